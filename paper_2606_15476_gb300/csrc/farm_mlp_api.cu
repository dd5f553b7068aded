// farm_mlp_api.cu -- the learned descriptor prefilter: weights, training on
// the GPU, loss/gradient evaluation, and tensor-core inference.
//
// f(x) = normalize(W2 gelu(W1 x + b1) + b2) maps a unit descriptor or query
// row (length D) to a unit vector of length P (128 by default).  Trained on
// (query row, object descriptor, oracle cosine y) pairs with the weighted
// squared error of f(q).f(d) against y, it replaces the full-length similarity
// stage by a P-length one whose best candidates are then re-scored exactly in
// FP32 (the plain full-descriptor path stays the fallback and the judge of
// its recall).  Training runs every contraction of the forward and backward
// passes as BF16 tensor-core products with FP32 accumulation (FP32 master
// weights, Adam); inference runs both layers the same way.  The FP32
// CUDA-core forward and backward are the reference arithmetic of
// farm_mlp_loss_grad and farm_mlp_embed.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "farm_internal.h"

using farm::Ctx;
using farm::Mlp;

namespace {

farm_status fail(Ctx &c, farm_status st, const std::string &msg)
{
    c.err = msg;
    return st;
}

#define MCK(call)                                                                                  \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess)                                                                     \
            return fail(c, e_ == cudaErrorMemoryAllocation ? FARM_ENOMEM : FARM_ECUDA,             \
                        std::string(#call) + ": " + cudaGetErrorString(e_));                       \
    } while (0)

#define MLAUNCH(call)     \
    do {                  \
        c.launches += 1;  \
        MCK(call);        \
    } while (0)

constexpr int64_t kEmbedChunk = 16384;   // rows per inference chunk

// SplitMix64 (Steele, Lea, Flood 2014) for the per-epoch shuffle.
uint64_t splitmix64(uint64_t &x)
{
    uint64_t z = (x += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Device scratch for training and loss/gradient evaluation (one allocation).
struct TrainBufs {
    float *base = nullptr;
    float *xq, *xd, *hq, *hd, *aq, *ad, *zq, *zd, *eq, *ed, *nq, *nd, *da, *grad, *m, *v, *loss, *y, *w;
};

cudaError_t train_alloc(TrainBufs &t, const Mlp &M, int64_t B, int64_t loss_slots)
{
    const int64_t D = M.D, H = M.H, P = M.P, cnt = M.count();
    const int64_t sizes[] = {B * D, B * D, B * H, B * H, B * H, B * H, B * P, B * P, B * P, B * P,
                             B,     B,     B * H, cnt,   cnt,   cnt,   loss_slots, B, B};
    float **dst[] = {&t.xq, &t.xd, &t.hq, &t.hd, &t.aq, &t.ad, &t.zq, &t.zd, &t.eq, &t.ed,
                     &t.nq, &t.nd, &t.da, &t.grad, &t.m, &t.v, &t.loss, &t.y, &t.w};
    auto rounded = [](int64_t n) { return (n + 63) / 64 * 64; };   // 256-byte aligned sub-arrays
    int64_t total = 0;
    for (int64_t n : sizes) total += rounded(n);
    cudaError_t e = cudaMalloc(&t.base, (size_t)total * sizeof(float));
    if (e != cudaSuccess) return e;
    float *p = t.base;
    for (size_t i = 0; i < sizeof(sizes) / sizeof(sizes[0]); ++i) {
        *dst[i] = p;
        p += rounded(sizes[i]);
    }
    return cudaSuccess;
}

// Forward of b rows X [b, D] (lda D): h, a, z kept, e = f(X), norm.
cudaError_t forward(const Mlp &M, const float *X, int64_t b, float *h, float *a, float *z, float *e, float *nrm,
                    cudaStream_t s, int64_t &launches)
{
    cudaError_t r;
    launches += 4;
    if ((r = farm::mlp_gemm(false, false, (int)b, M.H, M.D, 1.f, X, M.D, M.W1(), M.D, 0.f, h, M.H, s))) return r;
    if ((r = farm::mlp_bias_gelu(h, M.b1(), a, b, M.H, s))) return r;
    if ((r = farm::mlp_gemm(false, false, (int)b, M.P, M.H, 1.f, a, M.H, M.W2(), M.H, 0.f, z, M.P, s))) return r;
    return farm::mlp_bias_normalize(z, M.b2(), e, nrm, b, M.P, s);
}

// Backward of one tower given de (overwritten) into grad (beta 0: set, 1: add).
cudaError_t backward(const Mlp &M, const float *X, int64_t b, float *h, const float *a, const float *e,
                     const float *nrm, float *de, float *da, float *grad, float beta, cudaStream_t s,
                     int64_t &launches)
{
    const int64_t D = M.D, H = M.H, P = M.P;
    float *gW1 = grad, *gb1 = grad + H * D, *gW2 = gb1 + H, *gb2 = gW2 + P * H;
    cudaError_t r;
    launches += 8;
    if ((r = farm::mlp_normalize_backward(e, nrm, de, b, (int)P, s))) return r;
    if ((r = farm::mlp_gemm(true, true, (int)P, (int)H, (int)b, 1.f, de, (int)P, a, (int)H, beta, gW2, (int)H, s)))
        return r;
    if ((r = farm::mlp_colsum(de, b, (int)P, gb2, beta != 0.f, s))) return r;
    if ((r = farm::mlp_gemm(false, true, (int)b, (int)H, (int)P, 1.f, de, (int)P, M.W2(), (int)H, 0.f, da, (int)H, s)))
        return r;
    if ((r = farm::mlp_gelu_backward(h, da, b * H, s))) return r;
    if ((r = farm::mlp_gemm(true, true, (int)H, (int)D, (int)b, 1.f, da, (int)H, X, (int)D, beta, gW1, (int)D, s)))
        return r;
    return farm::mlp_colsum(da, b, (int)H, gb1, beta != 0.f, s);
}

// BF16 copies of the weights for the tensor-core products: W1 padded to D_pad
// columns, W2, and W2 transposed ([H, P], the operand of the backward pass).
cudaError_t refresh_bf16_weights(Ctx &c)
{
    Mlp &M = c.mlp;
    cudaError_t e = farm::mlp_to_bf16_padded(M.W1(), M.H, M.D, M.w1b, M.D_pad, c.stream);
    if (e == cudaSuccess) e = farm::mlp_to_bf16(M.W2(), (int64_t)M.P * M.H, M.w2b, c.stream);
    if (e == cudaSuccess) e = farm::mlp_transpose_bf16(M.W2(), nullptr, M.H, M.P, M.H, M.w2t, M.P, 0, c.stream);
    c.launches += 3;
    M.version += 1;
    return e;
}

// Device buffers of one tensor-core training step over up to B pairs: the
// two towers' rows are stacked (query rows 0..b-1, descriptor rows b..2b-1),
// so each contraction is one launch over 2b rows; the weight gradients
// contract over those 2b rows (K), padded with zero columns to a multiple of 64.
struct TcBufs {
    void *base = nullptr;
    int64_t B = 0, K_pad = 0;
    uint16_t *x, *ab, *dzb, *xT, *aT, *dzT, *dhT;
    float *h, *a, *z, *e, *nrm, *dz, *da, *grad, *m, *v, *loss, *y, *w;
};

int64_t round64(int64_t x) { return (x + 63) / 64 * 64; }

cudaError_t tc_alloc(TcBufs &t, const Mlp &M, int64_t B, int64_t loss_slots)
{
    const int64_t R = 2 * B, K = round64(2 * B), D = M.D, Dp = M.D_pad, H = M.H, P = M.P, cnt = M.count();
    t.B = B;
    t.K_pad = K;
    // (element count, element bytes) of each array, 256-byte aligned in one allocation
    const int64_t n16[] = {R * Dp, R * H, R * P, Dp * K, H * K, P * K, H * K};
    uint16_t **d16[] = {&t.x, &t.ab, &t.dzb, &t.xT, &t.aT, &t.dzT, &t.dhT};
    const int64_t n32[] = {R * H, R * H, R * P, R * P, R, R * P, R * H, cnt, cnt, cnt, loss_slots, B, B};
    float **d32[] = {&t.h, &t.a, &t.z, &t.e, &t.nrm, &t.dz, &t.da, &t.grad, &t.m, &t.v, &t.loss, &t.y, &t.w};
    (void)D;
    auto al = [](int64_t bytes) { return (bytes + 255) / 256 * 256; };
    int64_t total = 0;
    for (int64_t n : n16) total += al(n * 2);
    for (int64_t n : n32) total += al(n * 4);
    cudaError_t e = cudaMalloc(&t.base, (size_t)total);
    if (e != cudaSuccess) return e;
    char *p = static_cast<char *>(t.base);
    for (size_t i = 0; i < sizeof(n16) / sizeof(n16[0]); ++i) { *d16[i] = reinterpret_cast<uint16_t *>(p); p += al(n16[i] * 2); }
    for (size_t i = 0; i < sizeof(n32) / sizeof(n32[0]); ++i) { *d32[i] = reinterpret_cast<float *>(p); p += al(n32[i] * 4); }
    // the padding columns of the transposed operands stay zero unless a step writes them
    return cudaMemsetAsync(t.base, 0, (size_t)total);
}

// Loss and gradient of b pairs whose stacked BF16 input rows (query rows,
// then descriptor rows, D_pad long) are in t.x; targets / weights t.y, t.w
// (device, b each; w null: 1), wsum their sum.  The loss is added to *lslot,
// the gradient [W1 | b1 | W2 | b2] written to t.grad.
cudaError_t tc_loss_grad(Ctx &c, TcBufs &t, int64_t b, bool weighted, float wsum, float *lslot, int64_t &launches)
{
    const Mlp &M = c.mlp;
    const int64_t R = 2 * b, K = t.K_pad, H = M.H, P = M.P, D = M.D;
    float *gW1 = t.grad, *gb1 = gW1 + H * D, *gW2 = gb1 + H, *gb2 = gW2 + P * H;
    cudaStream_t st = c.stream;
    cudaError_t r;
    // zero the padding columns [R, K) of the transposed operands (rows of K entries)
    if (R < K) {
        uint16_t *tr[] = {t.xT, t.aT, t.dzT, t.dhT};
        const int64_t nr[] = {M.D_pad, H, P, H};
        for (int i = 0; i < 4; ++i)
            if ((r = cudaMemset2DAsync(tr[i] + R, (size_t)K * 2, 0, (size_t)(K - R) * 2, (size_t)nr[i], st)))
                return r;
    }
    launches += 17;
    // forward: h = x W1^T + b1, a = gelu(h), z = a W2^T + b2, e = z / |z|
    if ((r = farm::mlp_transpose_bf16(nullptr, t.x, M.D_pad, R, (int)D, t.xT, K, 0, st))) return r;
    if ((r = farm::launch_sim_tc_bf16(t.x, M.w1b, t.h, R, H, M.D_pad, H, nullptr, c.num_sms, c.d_err, st))) return r;
    if ((r = farm::mlp_bias_gelu(t.h, M.b1(), t.a, R, (int)H, st, t.ab))) return r;
    if ((r = farm::mlp_transpose_bf16(t.a, nullptr, H, R, (int)H, t.aT, K, 0, st))) return r;
    if ((r = farm::launch_sim_tc_bf16(t.ab, M.w2b, t.z, R, P, H, P, nullptr, c.num_sms, c.d_err, st))) return r;
    if ((r = farm::mlp_bias_normalize(t.z, M.b2(), t.e, t.nrm, R, (int)P, st))) return r;
    // loss; de of both towers
    if ((r = farm::mlp_pair_loss(t.e, t.e + b * P, t.y, weighted ? t.w : nullptr, wsum, b, (int)P, t.dz,
                                 t.dz + b * P, lslot, st)))
        return r;
    // backward: dz, gb2, dW2 = dz^T a, da = dz W2, dh = gelu'(h) da, gb1, dW1 = dh^T x
    if ((r = farm::mlp_normalize_backward(t.e, t.nrm, t.dz, R, (int)P, st))) return r;
    if ((r = farm::mlp_colsum(t.dz, R, (int)P, gb2, false, st))) return r;
    if ((r = farm::mlp_to_bf16(t.dz, R * P, t.dzb, st))) return r;
    if ((r = farm::mlp_transpose_bf16(t.dz, nullptr, P, R, (int)P, t.dzT, K, 0, st))) return r;
    if ((r = farm::launch_sim_tc_bf16(t.dzT, t.aT, gW2, P, H, K, H, nullptr, c.num_sms, c.d_err, st))) return r;
    if ((r = farm::launch_sim_tc_bf16(t.dzb, M.w2t, t.da, R, H, P, H, nullptr, c.num_sms, c.d_err, st))) return r;
    if ((r = farm::mlp_gelu_backward(t.h, t.da, R * H, st))) return r;
    if ((r = farm::mlp_colsum(t.da, R, (int)H, gb1, false, st))) return r;
    if ((r = farm::mlp_transpose_bf16(t.da, nullptr, H, R, (int)H, t.dhT, K, 0, st))) return r;
    return farm::launch_sim_tc_bf16(t.dhT, t.xT, gW1, H, D, K, D, nullptr, c.num_sms, c.d_err, st);
}

}  // namespace

namespace {

cudaError_t embed_buffers(farm_ctx *ctx, int64_t rows, void **h, void **a, void **ab, void **z, void **e)
{
    const Mlp &M = farm::ctx_of(ctx)->mlp;
    const int64_t chunk = std::max<int64_t>(1, std::min<int64_t>(rows, kEmbedChunk));
    cudaError_t r;
    if ((r = farm::ws_alloc(ctx, farm::B_MLP_H, (size_t)chunk * M.H * 4, h))) return r;
    if ((r = farm::ws_alloc(ctx, farm::B_MLP_A, (size_t)chunk * M.H * 4, a))) return r;
    if ((r = farm::ws_alloc(ctx, farm::B_MLP_AB, (size_t)chunk * M.H * 2, ab))) return r;
    if ((r = farm::ws_alloc(ctx, farm::B_MLP_Z, (size_t)chunk * M.P * 4, z))) return r;
    return farm::ws_alloc(ctx, farm::B_MLP_E, (size_t)chunk * M.P * 4, e);
}

}  // namespace

cudaError_t farm::learned_reserve(farm_ctx *ctx, int64_t rows)
{
    void *h, *a, *ab, *z, *e;
    return embed_buffers(ctx, rows, &h, &a, &ab, &z, &e);
}

cudaError_t farm::learned_embed_rows(farm_ctx *ctx, const uint16_t *xb, int64_t rows, uint16_t *out)
{
    Ctx &c = *ctx_of(ctx);
    const Mlp &M = c.mlp;
    const int64_t chunk = std::min<int64_t>(rows, kEmbedChunk);
    void *h, *a, *ab, *z, *e;
    cudaError_t r;
    if ((r = embed_buffers(ctx, rows, &h, &a, &ab, &z, &e))) return r;
    for (int64_t r0 = 0; r0 < rows; r0 += chunk) {
        const int64_t b = std::min(chunk, rows - r0);
        c.launches += 6;
        if ((r = launch_sim_tc_bf16(xb + r0 * M.D_pad, M.w1b, (float *)h, b, M.H, M.D_pad, M.H, nullptr, c.num_sms, c.d_err,
                                    c.stream)))
            return r;
        if ((r = mlp_bias_gelu((float *)h, M.b1(), (float *)a, b, M.H, c.stream))) return r;
        if ((r = mlp_to_bf16((float *)a, b * M.H, (uint16_t *)ab, c.stream))) return r;
        if ((r = launch_sim_tc_bf16((uint16_t *)ab, M.w2b, (float *)z, b, M.P, M.H, M.P, nullptr, c.num_sms, c.d_err,
                                    c.stream)))
            return r;
        if ((r = mlp_bias_normalize((float *)z, M.b2(), (float *)e, nullptr, b, M.P, c.stream))) return r;
        if ((r = mlp_to_bf16((float *)e, b * M.P, out + r0 * M.P, c.stream))) return r;
    }
    return cudaSuccess;
}

cudaError_t farm::learned_refresh_scene(farm_ctx *ctx, int32_t scene_id)
{
    Ctx &c = *ctx_of(ctx);
    Scene &s = c.scenes[scene_id];
    if (s.comp && s.comp_version == c.mlp.version) return cudaSuccess;
    cudaError_t r;
    if (!s.comp) {
        if ((r = cudaStreamSynchronize(c.stream))) return r;
        if ((r = cudaMalloc(&s.comp, (size_t)s.n * c.mlp.P * 2))) return r;
    }
    if ((r = learned_embed_rows(ctx, s.desc_bf16, s.n, s.comp))) return r;
    s.comp_version = c.mlp.version;
    return cudaSuccess;
}

extern "C" {

farm_status farm_mlp_set(farm_ctx *ctx, int32_t dim, int32_t hidden, int32_t out_dim, const float *W1,
                         const float *b1, const float *W2, const float *b2)
{
    if (!ctx) return FARM_EINVAL;
    Ctx &c = *farm::ctx_of(ctx);
    if (dim < 1 || dim > 8192 || hidden < 64 || hidden > 4096 || hidden % 64 || out_dim < 64 || out_dim > 1024 ||
        out_dim % 64)
        return fail(c, FARM_EINVAL, "farm_mlp_set: need 1 <= dim <= 8192, hidden in [64, 4096] and out_dim in "
                                    "[64, 1024], both multiples of 64");
    if (!W1 || !b1 || !W2 || !b2) return fail(c, FARM_EINVAL, "farm_mlp_set: weights must be non-null");
    MCK(cudaSetDevice(c.device));
    Mlp &M = c.mlp;
    Mlp nm;
    nm.D = dim; nm.H = hidden; nm.P = out_dim;
    nm.D_pad = (dim + farm::kDimAlign - 1) / farm::kDimAlign * farm::kDimAlign;
    const int64_t cnt = nm.count();
    std::vector<float> host((size_t)cnt);
    std::memcpy(host.data(), W1, (size_t)nm.H * nm.D * 4);
    std::memcpy(host.data() + (size_t)nm.H * nm.D, b1, (size_t)nm.H * 4);
    std::memcpy(host.data() + (size_t)nm.H * nm.D + nm.H, W2, (size_t)nm.P * nm.H * 4);
    std::memcpy(host.data() + (size_t)nm.H * nm.D + nm.H + (size_t)nm.P * nm.H, b2, (size_t)nm.P * 4);
    for (float x : host)
        if (!std::isfinite(x)) return fail(c, FARM_EINVAL, "farm_mlp_set: non-finite weight");
    MCK(cudaStreamSynchronize(c.stream));
    if (M.set && (M.D != nm.D || M.H != nm.H || M.P != nm.P)) {
        cudaFree(M.params); cudaFree(M.w1b); cudaFree(M.w2b); cudaFree(M.w2t);
        M.params = nullptr; M.w1b = nullptr; M.w2b = nullptr; M.w2t = nullptr;
        M.set = false;
    }
    if (!M.set) {
        MCK(cudaMalloc(&M.params, (size_t)cnt * 4));
        MCK(cudaMalloc(&M.w1b, (size_t)nm.H * nm.D_pad * 2));
        MCK(cudaMalloc(&M.w2b, (size_t)nm.P * nm.H * 2));
        MCK(cudaMalloc(&M.w2t, (size_t)nm.H * nm.P * 2));
        M.D = nm.D; M.H = nm.H; M.P = nm.P; M.D_pad = nm.D_pad;
        // shape change: every scene cache is stale
        for (auto &s : c.scenes)
            if (s.comp) { cudaFree(s.comp); s.comp = nullptr; }
    }
    MCK(cudaMemcpyAsync(M.params, host.data(), (size_t)cnt * 4, cudaMemcpyHostToDevice, c.stream));
    M.set = true;
    MCK(refresh_bf16_weights(c));
    // the host copy above must have been read before `host` goes away
    MCK(cudaStreamSynchronize(c.stream));
    return FARM_OK;
}

farm_status farm_mlp_get(farm_ctx *ctx, float *W1, float *b1, float *W2, float *b2)
{
    if (!ctx) return FARM_EINVAL;
    Ctx &c = *farm::ctx_of(ctx);
    const Mlp &M = c.mlp;
    if (!M.set) return fail(c, FARM_ESTATE, "farm_mlp_get: no weights set");
    MCK(cudaSetDevice(c.device));
    if (W1) MCK(cudaMemcpyAsync(W1, M.W1(), (size_t)M.H * M.D * 4, cudaMemcpyDeviceToHost, c.stream));
    if (b1) MCK(cudaMemcpyAsync(b1, M.b1(), (size_t)M.H * 4, cudaMemcpyDeviceToHost, c.stream));
    if (W2) MCK(cudaMemcpyAsync(W2, M.W2(), (size_t)M.P * M.H * 4, cudaMemcpyDeviceToHost, c.stream));
    if (b2) MCK(cudaMemcpyAsync(b2, M.b2(), (size_t)M.P * 4, cudaMemcpyDeviceToHost, c.stream));
    MCK(cudaStreamSynchronize(c.stream));
    return FARM_OK;
}

farm_status farm_mlp_loss_grad(farm_ctx *ctx, int64_t n_pairs, const float *xq, const float *xd, const float *y,
                               const float *w, int32_t precision, float *loss, float *grad)
{
    if (!ctx) return FARM_EINVAL;
    Ctx &c = *farm::ctx_of(ctx);
    const Mlp &M = c.mlp;
    if (!M.set) return fail(c, FARM_ESTATE, "farm_mlp_loss_grad: no weights set");
    if (n_pairs < 1 || n_pairs > (1 << 20) || !xq || !xd || !y || !loss)
        return fail(c, FARM_EINVAL, "farm_mlp_loss_grad: bad arguments");
    if (precision != FARM_PREC_FP32_SIMT && precision != FARM_PREC_BF16)
        return fail(c, FARM_EINVAL, "farm_mlp_loss_grad: precision must be FARM_PREC_FP32_SIMT or FARM_PREC_BF16");
    MCK(cudaSetDevice(c.device));
    double wsum = 0.0;
    for (int64_t i = 0; i < n_pairs; ++i) wsum += w ? (double)w[i] : 1.0;
    if (!(wsum > 0.0)) return fail(c, FARM_EINVAL, "farm_mlp_loss_grad: weights sum to zero");
    const size_t xb = (size_t)n_pairs * M.D * 4;
    int64_t L = 0;
    cudaError_t e = cudaSuccess;
    if (precision == FARM_PREC_BF16) {
        // the training step's arithmetic: stacked rows in BF16, tensor-core contractions
        TcBufs t;
        float *raw = nullptr;
        MCK(tc_alloc(t, M, n_pairs, 1));
        auto done = [&](farm_status st) { cudaStreamSynchronize(c.stream); cudaFree(t.base); cudaFree(raw); return st; };
        if (!e) e = cudaMalloc(&raw, 2 * xb);
        if (!e) e = cudaMemcpyAsync(raw, xq, xb, cudaMemcpyHostToDevice, c.stream);
        if (!e) e = cudaMemcpyAsync(raw + (size_t)n_pairs * M.D, xd, xb, cudaMemcpyHostToDevice, c.stream);
        if (!e) e = cudaMemcpyAsync(t.y, y, (size_t)n_pairs * 4, cudaMemcpyHostToDevice, c.stream);
        if (!e && w) e = cudaMemcpyAsync(t.w, w, (size_t)n_pairs * 4, cudaMemcpyHostToDevice, c.stream);
        if (!e) e = cudaMemsetAsync(t.loss, 0, 4, c.stream);
        if (!e) e = farm::mlp_to_bf16_padded(raw, 2 * n_pairs, M.D, t.x, M.D_pad, c.stream);
        if (!e) e = tc_loss_grad(c, t, n_pairs, w != nullptr, (float)wsum, t.loss, L);
        if (!e) e = cudaMemcpyAsync(loss, t.loss, 4, cudaMemcpyDeviceToHost, c.stream);
        if (!e && grad) e = cudaMemcpyAsync(grad, t.grad, (size_t)M.count() * 4, cudaMemcpyDeviceToHost, c.stream);
        if (!e) e = cudaStreamSynchronize(c.stream);
        c.launches += L + 1;
        if (e) return done(fail(c, FARM_ECUDA, std::string("farm_mlp_loss_grad: ") + cudaGetErrorString(e)));
        return done(FARM_OK);
    }
    TrainBufs t;
    MCK(train_alloc(t, M, n_pairs, 1));
    auto done = [&](farm_status st) { cudaFree(t.base); return st; };
    if (!e) e = cudaMemcpyAsync(t.xq, xq, xb, cudaMemcpyHostToDevice, c.stream);
    if (!e) e = cudaMemcpyAsync(t.xd, xd, xb, cudaMemcpyHostToDevice, c.stream);
    if (!e) e = cudaMemcpyAsync(t.y, y, (size_t)n_pairs * 4, cudaMemcpyHostToDevice, c.stream);
    if (!e && w) e = cudaMemcpyAsync(t.w, w, (size_t)n_pairs * 4, cudaMemcpyHostToDevice, c.stream);
    if (!e) e = cudaMemsetAsync(t.loss, 0, 4, c.stream);
    if (!e) e = forward(M, t.xq, n_pairs, t.hq, t.aq, t.zq, t.eq, t.nq, c.stream, L);
    if (!e) e = forward(M, t.xd, n_pairs, t.hd, t.ad, t.zd, t.ed, t.nd, c.stream, L);
    // de of both towers into zq / zd (the pre-normalisation values are no longer needed)
    if (!e) e = farm::mlp_pair_loss(t.eq, t.ed, t.y, w ? t.w : nullptr, (float)wsum, n_pairs, M.P, t.zq, t.zd,
                                    t.loss, c.stream);
    if (!e) e = backward(M, t.xq, n_pairs, t.hq, t.aq, t.eq, t.nq, t.zq, t.da, t.grad, 0.f, c.stream, L);
    if (!e) e = backward(M, t.xd, n_pairs, t.hd, t.ad, t.ed, t.nd, t.zd, t.da, t.grad, 1.f, c.stream, L);
    if (!e) e = cudaMemcpyAsync(loss, t.loss, 4, cudaMemcpyDeviceToHost, c.stream);
    if (!e && grad) e = cudaMemcpyAsync(grad, t.grad, (size_t)M.count() * 4, cudaMemcpyDeviceToHost, c.stream);
    if (!e) e = cudaStreamSynchronize(c.stream);
    c.launches += L + 1;
    if (e) return done(fail(c, FARM_ECUDA, std::string("farm_mlp_loss_grad: ") + cudaGetErrorString(e)));
    return done(FARM_OK);
}

farm_status farm_mlp_train(farm_ctx *ctx, int32_t n_scenes, const int32_t *scene_ids, int64_t n_rows,
                           const float *rows, int64_t n_pairs, const int32_t *pair_row, const int32_t *pair_scene,
                           const int32_t *pair_obj, const float *y, const float *w, int32_t epochs, int32_t batch,
                           float lr, uint64_t seed, float *loss_out)
{
    if (!ctx) return FARM_EINVAL;
    Ctx &c = *farm::ctx_of(ctx);
    Mlp &M = c.mlp;
    if (!M.set) return fail(c, FARM_ESTATE, "farm_mlp_train: set initial weights with farm_mlp_set first");
    if (n_scenes < 1 || n_scenes > 64 || !scene_ids || (n_scenes > 1 && !pair_scene))
        return fail(c, FARM_EINVAL, "farm_mlp_train: need 1..64 scene ids (and pair_scene for more than one)");
    std::vector<const uint16_t *> bases((size_t)n_scenes + 1);   // the scenes' BF16 descriptors, then the rows
    std::vector<int64_t> scene_n((size_t)n_scenes);
    for (int32_t k = 0; k < n_scenes; ++k) {
        const int32_t sid = scene_ids[k];
        if (sid < 0 || sid >= (int32_t)c.scenes.size() || !c.scenes[sid].present)
            return fail(c, FARM_EINVAL, "farm_mlp_train: unknown scene");
        const farm::Scene &s = c.scenes[sid];
        if (s.dim != M.D) return fail(c, FARM_EINVAL, "farm_mlp_train: scene dim differs from the network's");
        bases[k] = s.desc_bf16;
        scene_n[k] = s.n;
    }
    if (n_rows < 1 || !rows || n_pairs < 1 || !pair_row || !pair_obj || !y || epochs < 1 || batch < 1 ||
        batch > (1 << 16) || !(lr > 0.f))
        return fail(c, FARM_EINVAL, "farm_mlp_train: bad arguments");
    for (int64_t i = 0; i < n_pairs; ++i) {
        const int32_t k = pair_scene ? pair_scene[i] : 0;
        if (pair_row[i] < 0 || pair_row[i] >= n_rows || k < 0 || k >= n_scenes || pair_obj[i] < 0 ||
            pair_obj[i] >= scene_n[k] || !std::isfinite(y[i]) || (w && !(w[i] >= 0.f)))
            return fail(c, FARM_EINVAL, "farm_mlp_train: pair " + std::to_string(i) + " out of range");
    }
    MCK(cudaSetDevice(c.device));
    const int64_t B = std::min<int64_t>(batch, n_pairs);
    const int64_t steps = (n_pairs + B - 1) / B;
    TcBufs t;
    MCK(tc_alloc(t, M, B, steps * (int64_t)epochs));
    uint16_t *qnb = nullptr;   // normalised training rows, BF16 [n_rows, D_pad]
    float *raw = nullptr;
    int32_t *d_idx = nullptr;  // per epoch: query rows [n_pairs] | object indices [n_pairs] | scenes [n_pairs]
    float *d_yw = nullptr;     // per epoch: targets [n_pairs] | weights [n_pairs]
    const uint16_t **d_bases = nullptr;
    auto done = [&](farm_status st) {
        cudaStreamSynchronize(c.stream);
        cudaFree(t.base); cudaFree(qnb); cudaFree(raw); cudaFree(d_idx); cudaFree(d_yw); cudaFree(d_bases);
        return st;
    };
    cudaError_t e = cudaSuccess;
    if (!e) e = cudaMalloc(&qnb, (size_t)n_rows * M.D_pad * 2);
    if (!e) e = cudaMalloc(&raw, (size_t)n_rows * M.D * 4);
    if (!e) e = cudaMalloc(&d_idx, (size_t)n_pairs * 3 * 4);
    if (!e) e = cudaMalloc(&d_yw, (size_t)n_pairs * 2 * 4);
    bases[n_scenes] = qnb;
    if (!e) e = cudaMalloc(&d_bases, bases.size() * sizeof(void *));
    if (!e) e = cudaMemcpyAsync(d_bases, bases.data(), bases.size() * sizeof(void *), cudaMemcpyHostToDevice,
                                c.stream);
    if (!e) e = cudaMemcpyAsync(raw, rows, (size_t)n_rows * M.D * 4, cudaMemcpyHostToDevice, c.stream);
    if (!e) e = farm::launch_normalize_rows(raw, nullptr, n_rows, M.D, M.D_pad, nullptr, nullptr, nullptr, qnb,
                                            c.d_err, farm::kErrBadRow, c.stream);
    if (!e) e = cudaMemsetAsync(t.m, 0, (size_t)M.count() * 4, c.stream);
    if (!e) e = cudaMemsetAsync(t.v, 0, (size_t)M.count() * 4, c.stream);
    if (!e) e = cudaMemsetAsync(t.loss, 0, (size_t)steps * epochs * 4, c.stream);
    if (e) return done(fail(c, FARM_ECUDA, std::string("farm_mlp_train: ") + cudaGetErrorString(e)));
    std::vector<int32_t> perm((size_t)n_pairs), hidx((size_t)n_pairs * 3);
    std::vector<float> hyw((size_t)n_pairs * 2);
    for (int64_t i = 0; i < n_pairs; ++i) perm[i] = (int32_t)i;
    uint64_t st = seed;
    int64_t L = 2;
    int t_adam = 0;
    for (int32_t ep = 0; ep < epochs && !e; ++ep) {
        for (int64_t i = n_pairs - 1; i > 0; --i) {
            const int64_t j = (int64_t)(splitmix64(st) % (uint64_t)(i + 1));
            std::swap(perm[i], perm[j]);
        }
        for (int64_t i = 0; i < n_pairs; ++i) {
            hidx[i] = pair_row[perm[i]];
            hidx[n_pairs + i] = pair_obj[perm[i]];
            hidx[2 * n_pairs + i] = pair_scene ? pair_scene[perm[i]] : 0;
            hyw[i] = y[perm[i]];
            hyw[n_pairs + i] = w ? w[perm[i]] : 1.f;
        }
        // the previous epoch's kernels may still read the device copies
        e = cudaStreamSynchronize(c.stream);
        if (!e) e = cudaMemcpyAsync(d_idx, hidx.data(), hidx.size() * 4, cudaMemcpyHostToDevice, c.stream);
        if (!e) e = cudaMemcpyAsync(d_yw, hyw.data(), hyw.size() * 4, cudaMemcpyHostToDevice, c.stream);
        for (int64_t sidx = 0; sidx < steps && !e; ++sidx) {
            const int64_t off = sidx * B;
            const int64_t b = std::min(B, n_pairs - off);
            double wsum = 0.0;
            for (int64_t i = 0; i < b; ++i) wsum += hyw[n_pairs + off + i];
            if (!(wsum > 0.0)) continue;
            float *lslot = t.loss + (int64_t)ep * steps + sidx;
            // stacked input rows: the pairs' query rows, then their descriptors
            L += 2;
            e = farm::mlp_gather_rows_bf16(d_bases + n_scenes, nullptr, d_idx + off, M.D_pad, b, M.D_pad, t.x,
                                           M.D_pad, c.stream);
            if (!e) e = farm::mlp_gather_rows_bf16(d_bases, d_idx + 2 * n_pairs + off, d_idx + n_pairs + off, M.D_pad,
                                                   b, M.D_pad, t.x + b * M.D_pad, M.D_pad, c.stream);
            if (!e) e = cudaMemcpyAsync(t.y, d_yw + off, (size_t)b * 4, cudaMemcpyDeviceToDevice, c.stream);
            if (!e) e = cudaMemcpyAsync(t.w, d_yw + n_pairs + off, (size_t)b * 4, cudaMemcpyDeviceToDevice, c.stream);
            if (!e) e = tc_loss_grad(c, t, b, true, (float)wsum, lslot, L);
            if (!e) e = farm::mlp_adam(M.params, t.grad, t.m, t.v, M.count(), lr, ++t_adam, c.stream);
            if (!e) e = refresh_bf16_weights(c);
            L += 1;
        }
    }
    c.launches += L;
    if (!e && loss_out) {
        std::vector<float> ls((size_t)steps * epochs);
        e = cudaMemcpyAsync(ls.data(), t.loss, ls.size() * 4, cudaMemcpyDeviceToHost, c.stream);
        if (!e) e = cudaStreamSynchronize(c.stream);
        for (int32_t ep = 0; ep < epochs && !e; ++ep) {
            double acc = 0.0;
            for (int64_t i = 0; i < steps; ++i) acc += ls[(size_t)ep * steps + i];
            loss_out[ep] = (float)(acc / (double)steps);
        }
    }
    if (e) return done(fail(c, FARM_ECUDA, std::string("farm_mlp_train: ") + cudaGetErrorString(e)));
    return done(FARM_OK);
}

farm_status farm_mlp_embed(farm_ctx *ctx, int64_t n_rows, const float *x, int32_t precision, float *out)
{
    if (!ctx) return FARM_EINVAL;
    Ctx &c = *farm::ctx_of(ctx);
    const Mlp &M = c.mlp;
    if (!M.set) return fail(c, FARM_ESTATE, "farm_mlp_embed: no weights set");
    if (n_rows < 0 || (n_rows > 0 && (!x || !out))) return fail(c, FARM_EINVAL, "farm_mlp_embed: bad arguments");
    if (precision != FARM_PREC_FP32_SIMT && precision != FARM_PREC_BF16)
        return fail(c, FARM_EINVAL, "farm_mlp_embed: precision must be FARM_PREC_FP32_SIMT or FARM_PREC_BF16");
    if (n_rows == 0) return FARM_OK;
    MCK(cudaSetDevice(c.device));
    float *raw = nullptr, *xn = nullptr, *h = nullptr, *a = nullptr, *z = nullptr, *e32 = nullptr;
    uint16_t *xb = nullptr, *eb = nullptr;
    auto done = [&](farm_status st) {
        cudaStreamSynchronize(c.stream);
        cudaFree(raw); cudaFree(xn); cudaFree(h); cudaFree(a); cudaFree(z); cudaFree(e32); cudaFree(xb); cudaFree(eb);
        return st;
    };
    cudaError_t e = cudaMalloc(&raw, (size_t)n_rows * M.D * 4);
    if (!e) e = cudaMemcpyAsync(raw, x, (size_t)n_rows * M.D * 4, cudaMemcpyHostToDevice, c.stream);
    if (precision == FARM_PREC_FP32_SIMT) {
        if (!e) e = cudaMalloc(&xn, (size_t)n_rows * M.D * 4);
        if (!e) e = cudaMalloc(&h, (size_t)n_rows * M.H * 4);
        if (!e) e = cudaMalloc(&a, (size_t)n_rows * M.H * 4);
        if (!e) e = cudaMalloc(&z, (size_t)n_rows * M.P * 4);
        if (!e) e = cudaMalloc(&e32, (size_t)n_rows * M.P * 4);
        if (!e) e = farm::launch_normalize_rows(raw, nullptr, n_rows, M.D, M.D, xn, nullptr, nullptr, nullptr, c.d_err,
                                                farm::kErrBadRow, c.stream);
        int64_t L = 1;
        if (!e) e = forward(M, xn, n_rows, h, a, z, e32, nullptr, c.stream, L);
        c.launches += L;
        if (!e) e = cudaMemcpyAsync(out, e32, (size_t)n_rows * M.P * 4, cudaMemcpyDeviceToHost, c.stream);
    } else {
        if (!e) e = cudaMalloc(&xb, (size_t)n_rows * M.D_pad * 2);
        if (!e) e = cudaMalloc(&eb, (size_t)n_rows * M.P * 2);
        if (!e) e = cudaMalloc(&e32, (size_t)n_rows * M.P * 4);
        if (!e) e = farm::launch_normalize_rows(raw, nullptr, n_rows, M.D, M.D_pad, nullptr, nullptr, nullptr, xb,
                                                c.d_err, farm::kErrBadRow, c.stream);
        c.launches += 1;
        if (!e) e = farm::learned_embed_rows(ctx, xb, n_rows, eb);
        // widen the BF16 embeddings for the caller
        std::vector<uint16_t> hb;
        if (!e) {
            hb.resize((size_t)n_rows * M.P);
            e = cudaMemcpyAsync(hb.data(), eb, hb.size() * 2, cudaMemcpyDeviceToHost, c.stream);
        }
        if (!e) e = cudaStreamSynchronize(c.stream);
        if (!e)
            for (size_t i = 0; i < hb.size(); ++i) {
                const uint32_t u = (uint32_t)hb[i] << 16;
                std::memcpy(out + i, &u, 4);
            }
    }
    if (!e) e = cudaStreamSynchronize(c.stream);
    if (e) return done(fail(c, FARM_ECUDA, std::string("farm_mlp_embed: ") + cudaGetErrorString(e)));
    farm_status st = FARM_OK;
    if (c.h_err) {
        cudaMemcpy(c.h_err, c.d_err, 4, cudaMemcpyDeviceToHost);
        if (*c.h_err) {
            cudaMemset(c.d_err, 0, 4);
            st = fail(c, FARM_EINVAL, "farm_mlp_embed: a row has zero or non-finite norm");
        }
    }
    return done(st);
}

}  // extern "C"
