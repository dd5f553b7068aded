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

// One call's device memory, freed when the call returns.
struct DevBufs {
    cudaStream_t stream = nullptr;
    std::vector<void *> ptrs;
    ~DevBufs()
    {
        if (stream) cudaStreamSynchronize(stream);    // no work of the call still uses them
        for (void *p : ptrs) cudaFree(p);
    }
    template <class T>
    cudaError_t get(T **out, size_t count)
    {
        void *p = nullptr;
        const cudaError_t e = cudaMalloc(&p, std::max<size_t>(count, 1) * sizeof(T));
        if (e == cudaSuccess) ptrs.push_back(p);
        *out = static_cast<T *>(p);
        return e;
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
    DevBufs db;
    db.stream = c.stream;
    // inputs on the device
    const float *d_emu = ent_mu, *d_ecov = ent_cov, *d_efeat = ent_feat, *d_ew = ent_w;
    const int32_t *d_eact = ent_active;
    const float *d_dmu = det_mu, *d_dcov = det_cov, *d_dfeat = det_feat;
    if (!dev) {
        float *p;
        int32_t *pi;
        const cudaMemcpyKind k = cudaMemcpyHostToDevice;
        ACK(db.get(&p, (size_t)3 * N), "alloc");
        ACK(cudaMemcpyAsync(p, ent_mu, (size_t)3 * N * 4, k, c.stream), "copy");
        d_emu = p;
        ACK(db.get(&p, (size_t)6 * N), "alloc");
        ACK(cudaMemcpyAsync(p, ent_cov, (size_t)6 * N * 4, k, c.stream), "copy");
        d_ecov = p;
        ACK(db.get(&p, (size_t)N * F), "alloc");
        ACK(cudaMemcpyAsync(p, ent_feat, (size_t)N * F * 4, k, c.stream), "copy");
        d_efeat = p;
        ACK(db.get(&p, (size_t)N), "alloc");
        ACK(cudaMemcpyAsync(p, ent_w, (size_t)N * 4, k, c.stream), "copy");
        d_ew = p;
        ACK(db.get(&pi, (size_t)N), "alloc");
        ACK(cudaMemcpyAsync(pi, ent_active, (size_t)N * 4, k, c.stream), "copy");
        d_eact = pi;
        ACK(db.get(&p, (size_t)3 * B), "alloc");
        ACK(cudaMemcpyAsync(p, det_mu, (size_t)3 * B * 4, k, c.stream), "copy");
        d_dmu = p;
        ACK(db.get(&p, (size_t)6 * B), "alloc");
        ACK(cudaMemcpyAsync(p, det_cov, (size_t)6 * B * 4, k, c.stream), "copy");
        d_dcov = p;
        ACK(db.get(&p, (size_t)B * F), "alloc");
        ACK(cudaMemcpyAsync(p, det_feat, (size_t)B * F * 4, k, c.stream), "copy");
        d_dfeat = p;
    }
    // feature cosines: unit rows in the FP16 split, the FP32-accurate similarity kernel
    uint16_t *dhi, *dlo, *ehi, *elo;
    float *S;
    ACK(db.get(&dhi, (size_t)B * F_pad), "alloc");
    ACK(db.get(&dlo, (size_t)B * F_pad), "alloc");
    ACK(db.get(&ehi, (size_t)N * F_pad), "alloc");
    ACK(db.get(&elo, (size_t)N * F_pad), "alloc");
    ACK(db.get(&S, (size_t)B * ld), "alloc");
    c.launches += 3;
    ACK(farm::launch_normalize_rows(d_dfeat, nullptr, B, F, F_pad, nullptr, dhi, dlo, nullptr, c.d_err,
                                    farm::kErrBadRow, c.stream), "normalise detections");
    ACK(farm::launch_normalize_rows(d_efeat, nullptr, N, F, F_pad, nullptr, ehi, elo, nullptr, c.d_err,
                                    farm::kErrBadDesc, c.stream), "normalise entities");
    if (!farm::sim_tc_available()) return afail(c, FARM_EINVAL, "the tensor-core similarity path is not built");
    ACK(farm::launch_sim_tc_f16x3(dhi, dlo, ehi, elo, S, B, N, F_pad, ld, nullptr, c.num_sms, c.d_err, c.stream),
        "feature cosines");
    // search, components, fusion
    farm::AssocArgs a{};
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
    ACK(db.get(&a.label, (size_t)T), "alloc");
    ACK(db.get(&a.win, (size_t)T), "alloc");
    ACK(db.get(&a.acc, (size_t)T * (10 + F)), "alloc");
    if (dev) {
        a.match_cnt = match_cnt;
        a.match_idx = match_idx;
        a.match_h = match_h;
        a.parent = parent;
        a.out_w = out_w;
        a.out_mu = out_mu;
        a.out_cov = out_cov;
        a.out_feat = out_feat;
    } else {
        ACK(db.get(&a.match_cnt, (size_t)B), "alloc");
        ACK(db.get(&a.match_idx, (size_t)B * max_m), "alloc");
        ACK(db.get(&a.match_h, (size_t)B * max_m), "alloc");
        ACK(db.get(&a.parent, (size_t)T), "alloc");
        ACK(db.get(&a.out_w, (size_t)T), "alloc");
        ACK(db.get(&a.out_mu, (size_t)3 * T), "alloc");
        ACK(db.get(&a.out_cov, (size_t)6 * T), "alloc");
        ACK(db.get(&a.out_feat, (size_t)T * F), "alloc");
    }
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
    // the call's buffers are freed on return: wait for the work that uses them
    ACK(cudaStreamSynchronize(c.stream), "synchronise");
    return farm_sync(ctx);
#undef ACK
}
