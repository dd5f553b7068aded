// farm_assoc_api.cu -- farm_associate: the mapping-side association of a
// batch of detections with the memory's entities (App. D.1 steps 3-5; the
// kernels are in k_assoc.cu).
#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "farm_internal.h"

using farm::Ctx;

namespace {

farm_status afail(Ctx &c, farm_status st, const std::string &msg)
{
    c.err = msg;
    return st;
}

// Sub-arrays carved from the context's grow-only association buffer (each
// on a 256-byte boundary): a first pass sums the sizes, the second hands out
// pointers.
struct Carve {
    uint8_t *base = nullptr;
    size_t off = 0;
    template <class T>
    T *take(size_t count)
    {
        T *p = reinterpret_cast<T *>(base ? base + off : nullptr);
        off += (std::max<size_t>(count, 1) * sizeof(T) + 255) & ~size_t(255);
        return p;
    }
};

}  // namespace

extern "C" farm_status farm_associate(farm_ctx *ctx, int64_t n_ent, const float *ent_mu, const float *ent_cov,
                                      const float *ent_feat, const int32_t *ent_active, const float *ent_w,
                                      int64_t n_det, const float *det_mu, const float *det_cov, const float *det_feat,
                                      int32_t F, float tau_f, float h_max, int32_t max_m, int32_t *match_cnt,
                                      int32_t *match_idx, float *match_h, int32_t *parent, float *out_w,
                                      float *out_mu, float *out_cov, float *out_feat, uint32_t flags)
{
    if (!ctx) return FARM_EINVAL;
    Ctx &c = *farm::ctx_of(ctx);
    if (n_ent < 1 || n_det < 1 || n_ent + n_det > 0x7fffffff)
        return afail(c, FARM_EINVAL, "farm_associate: n_ent and n_det must be >= 1 (and their sum < 2^31)");
    if (F < 1 || F > 8192) return afail(c, FARM_EINVAL, "farm_associate: F must lie in [1, 8192]");
    if (max_m < 1 || max_m > 64) return afail(c, FARM_EINVAL, "farm_associate: max_m must lie in [1, 64]");
    if (!(tau_f >= -1.f && tau_f <= 1.f) || !(h_max >= 0.f && h_max <= 1.f))
        return afail(c, FARM_EINVAL, "farm_associate: tau_f must lie in [-1, 1] and h_max in [0, 1]");
    if (!ent_mu || !ent_cov || !ent_feat || !ent_active || !ent_w || !det_mu || !det_cov || !det_feat ||
        !match_cnt || !match_idx || !match_h || !parent || !out_w || !out_mu || !out_cov || !out_feat)
        return afail(c, FARM_EINVAL, "farm_associate: null array");
    const bool dev = (flags & FARM_PTR_DEVICE) != 0;
    if (!dev) {
        for (int64_t e = 0; e < n_ent; ++e)
            if (!(ent_w[e] >= 0.f) || !std::isfinite(ent_w[e]))
                return afail(c, FARM_EINVAL, "farm_associate: entity weights must be finite and >= 0");
    }
    const int32_t N = (int32_t)n_ent, B = (int32_t)n_det, T = N + B;
    const int32_t F_pad = (int32_t)((F + farm::kDimAlign - 1) / farm::kDimAlign * farm::kDimAlign);
    const int64_t ld = (N + 31) / 32 * 32;
    auto ck = [&](cudaError_t e, const char *what) -> farm_status {
        if (e == cudaSuccess) return FARM_OK;
        return afail(c, e == cudaErrorMemoryAllocation ? FARM_ENOMEM : FARM_ECUDA,
                     std::string("farm_associate: ") + what + ": " + cudaGetErrorString(e));
    };
#define ACK(call, what)                                \
    do {                                               \
        const farm_status st_ = ck((call), what);      \
        if (st_ != FARM_OK) return st_;                \
    } while (0)
    ACK(cudaSetDevice(c.device), "set device");
    farm::AssocArgs a{};
    const float *d_emu = ent_mu, *d_ecov = ent_cov, *d_efeat = ent_feat, *d_ew = ent_w;
    const int32_t *d_eact = ent_active;
    const float *d_dmu = det_mu, *d_dcov = det_cov, *d_dfeat = det_feat;
    uint16_t *dhi = nullptr, *dlo = nullptr, *ehi = nullptr, *elo = nullptr;
    float *S = nullptr;
    float *h_emu = nullptr, *h_ecov = nullptr, *h_efeat = nullptr, *h_ew = nullptr, *h_dmu = nullptr,
          *h_dcov = nullptr, *h_dfeat = nullptr;
    int32_t *h_eact = nullptr;
    // the layout of the call's device memory: sized with a null base, then
    // carved from the context's grow-only buffer
    auto layout = [&](Carve &cv) {
        if (!dev) {
            h_emu = cv.take<float>((size_t)3 * N); h_ecov = cv.take<float>((size_t)6 * N);
            h_efeat = cv.take<float>((size_t)N * F); h_ew = cv.take<float>((size_t)N);
            h_eact = cv.take<int32_t>((size_t)N); h_dmu = cv.take<float>((size_t)3 * B);
            h_dcov = cv.take<float>((size_t)6 * B); h_dfeat = cv.take<float>((size_t)B * F);
        }
        dhi = cv.take<uint16_t>((size_t)B * F_pad); dlo = cv.take<uint16_t>((size_t)B * F_pad);
        ehi = cv.take<uint16_t>((size_t)N * F_pad); elo = cv.take<uint16_t>((size_t)N * F_pad);
        S = cv.take<float>((size_t)B * ld);
        a.label = cv.take<int32_t>((size_t)T);
        a.win = cv.take<unsigned long long>((size_t)T);
        a.acc = cv.take<float>((size_t)T * (10 + F));
        if (dev) {
            a.match_cnt = match_cnt; a.match_idx = match_idx; a.match_h = match_h; a.parent = parent;
            a.out_w = out_w; a.out_mu = out_mu; a.out_cov = out_cov; a.out_feat = out_feat;
        } else {
            a.match_cnt = cv.take<int32_t>((size_t)B); a.match_idx = cv.take<int32_t>((size_t)B * max_m);
            a.match_h = cv.take<float>((size_t)B * max_m); a.parent = cv.take<int32_t>((size_t)T);
            a.out_w = cv.take<float>((size_t)T); a.out_mu = cv.take<float>((size_t)3 * T);
            a.out_cov = cv.take<float>((size_t)6 * T); a.out_feat = cv.take<float>((size_t)T * F);
        }
    };
    {
        Carve sizing;
        layout(sizing);
        void *buf = nullptr;
        ACK(farm::ws_alloc(ctx, farm::B_ASSOC, sizing.off, &buf), "workspace");
        Carve cv;
        cv.base = static_cast<uint8_t *>(buf);
        layout(cv);
    }
    if (!dev) {
        const cudaMemcpyKind k = cudaMemcpyHostToDevice;
        ACK(cudaMemcpyAsync(h_emu, ent_mu, (size_t)3 * N * 4, k, c.stream), "copy");
        ACK(cudaMemcpyAsync(h_ecov, ent_cov, (size_t)6 * N * 4, k, c.stream), "copy");
        ACK(cudaMemcpyAsync(h_efeat, ent_feat, (size_t)N * F * 4, k, c.stream), "copy");
        ACK(cudaMemcpyAsync(h_ew, ent_w, (size_t)N * 4, k, c.stream), "copy");
        ACK(cudaMemcpyAsync(h_eact, ent_active, (size_t)N * 4, k, c.stream), "copy");
        ACK(cudaMemcpyAsync(h_dmu, det_mu, (size_t)3 * B * 4, k, c.stream), "copy");
        ACK(cudaMemcpyAsync(h_dcov, det_cov, (size_t)6 * B * 4, k, c.stream), "copy");
        ACK(cudaMemcpyAsync(h_dfeat, det_feat, (size_t)B * F * 4, k, c.stream), "copy");
        d_emu = h_emu; d_ecov = h_ecov; d_efeat = h_efeat; d_ew = h_ew; d_eact = h_eact;
        d_dmu = h_dmu; d_dcov = h_dcov; d_dfeat = h_dfeat;
    }
    // feature cosines: unit rows in the FP16 split, the FP32-accurate similarity kernel
    c.launches += 3;
    ACK(farm::launch_normalize_rows(d_dfeat, nullptr, B, F, F_pad, nullptr, dhi, dlo, nullptr, c.d_err,
                                    farm::kErrBadRow, c.stream), "normalise detections");
    ACK(farm::launch_normalize_rows(d_efeat, nullptr, N, F, F_pad, nullptr, ehi, elo, nullptr, c.d_err,
                                    farm::kErrBadDesc, c.stream), "normalise entities");
    if (!farm::sim_tc_available()) return afail(c, FARM_EINVAL, "the tensor-core similarity path is not built");
    ACK(farm::launch_sim_tc_f16x3(dhi, dlo, ehi, elo, S, B, N, F_pad, ld, nullptr, c.num_sms, c.d_err, c.stream),
        "feature cosines");
    // search, components, fusion
    a.N = N;
    a.B = B;
    a.F = F;
    a.S = S;
    a.ld = ld;
    a.ent_mu = d_emu;
    a.ent_cov = d_ecov;
    a.ent_feat = d_efeat;
    a.ent_w = d_ew;
    a.ent_active = d_eact;
    a.det_mu = d_dmu;
    a.det_cov = d_dcov;
    a.det_feat = d_dfeat;
    a.tau_f = tau_f;
    a.h_max = h_max;
    a.max_m = max_m;
    a.err = c.d_err;
    c.launches += 9;
    ACK(farm::launch_assoc(a, c.stream), "association kernels");
    if (!dev) {
        const cudaMemcpyKind k = cudaMemcpyDeviceToHost;
        ACK(cudaMemcpyAsync(match_cnt, a.match_cnt, (size_t)B * 4, k, c.stream), "copy out");
        ACK(cudaMemcpyAsync(match_idx, a.match_idx, (size_t)B * max_m * 4, k, c.stream), "copy out");
        ACK(cudaMemcpyAsync(match_h, a.match_h, (size_t)B * max_m * 4, k, c.stream), "copy out");
        ACK(cudaMemcpyAsync(parent, a.parent, (size_t)T * 4, k, c.stream), "copy out");
        ACK(cudaMemcpyAsync(out_w, a.out_w, (size_t)T * 4, k, c.stream), "copy out");
        ACK(cudaMemcpyAsync(out_mu, a.out_mu, (size_t)3 * T * 4, k, c.stream), "copy out");
        ACK(cudaMemcpyAsync(out_cov, a.out_cov, (size_t)6 * T * 4, k, c.stream), "copy out");
        ACK(cudaMemcpyAsync(out_feat, a.out_feat, (size_t)T * F * 4, k, c.stream), "copy out");
    }
    if (dev) return FARM_OK;            // stream-ordered; errors at the next synchronising call
    ACK(cudaStreamSynchronize(c.stream), "synchronise");
    return farm_sync(ctx);
#undef ACK
}
