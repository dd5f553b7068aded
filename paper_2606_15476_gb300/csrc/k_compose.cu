// k_compose.cu -- relation evaluation, best-witness binding and composite
// scoring of every kept target candidate (App. D.2 steps 4-5; App. B).
//
// One CTA per query.  The query's landmark candidates (K_a per constraint,
// in rank order) and their centres are staged in shared memory.  For every
// kept target candidate of rank r the CTA computes
//   s_sem = cf / (mu + r)                       (cf = class_mis on a class mismatch)
// and the k_max-th largest s_sem, S_K.  k_max candidates score at least
// (1 - w) S_K, so a candidate with s_sem < (1 - w) S_K cannot enter any TopK of
// size <= k_max (its composite is at most s_sem); only the others are scored:
//   t_i   = max_{a in L_i, a != e} r_rho_i(e, a)   (bound anchor = argmax, lower index on ties)
//   gbar  = (prod_i t_i)^(1/m),  s = s_sem * ((1 - w) + w * gbar)
// with (candidate, constraint, landmark) triples spread over the threads and
// the best witness kept by a 64-bit atomic max over (r, ~index).  Because the
// composite is non-decreasing in every t_i and the anchors only meet at the
// target, the best binding takes each anchor's best witness on its own (the
// star decomposition of App. B).  The CTA then sorts the scored candidates by
// (s descending, object index ascending) so that any TopK is a prefix.
#include "farm_internal.h"

namespace farm {
namespace {

constexpr int TH = 256;

__device__ __forceinline__ float sigm(float x)
{
    if (x >= 0.f) return 1.f / (1.f + expf(-x));
    const float ex = expf(x);
    return ex / (1.f + ex);
}

__device__ __forceinline__ uint32_t order_key(float f)
{
    const uint32_t u = __float_as_uint(f + 0.0f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

// Left/right in the stored views of the candidate e (sign +1: LeftOf, -1: RightOf).
__device__ float viewpoint_lr(const float *__restrict__ ve, int n_views, float ex, float ey,
                              float ez, float ax, float ay, float az, float sign,
                              const farm_params &p)
{
    float acc = 0.f;
    int counted = 0;
    for (int v = 0; v < n_views; ++v) {
        const float4 o = *reinterpret_cast<const float4 *>(ve + v * kViewStride);
        const float4 f = *reinterpret_cast<const float4 *>(ve + v * kViewStride + 4);
        // o = (ox, oy, oz, fx), f = (fy, fz, rx, ry)
        const float fx = o.w, fy = f.x, fz = f.y, rx = f.z, ry = f.w;
        const float dex = ex - o.x, dey = ey - o.y, dez = ez - o.z;
        const float dax = ax - o.x, day = ay - o.y, daz = az - o.z;
        const float Ze = dex * fx + dey * fy + dez * fz;
        const float Za = dax * fx + day * fy + daz * fz;
        if (!(Ze > p.z_min && Za > p.z_min)) continue;
        const float ue = (dex * rx + dey * ry) / Ze;
        const float ua = (dax * rx + day * ry) / Za;
        acc += sigm(sign * (ua - ue) / p.tau_h);
        ++counted;
    }
    return counted ? acc / (float)counted : 0.5f;
}

__device__ __forceinline__ float relation(int pred, float ex, float ey, float ez, float ax,
                                          float ay, float az, const float *__restrict__ ve,
                                          int n_views, const farm_params &p)
{
    switch (pred) {
    case FARM_ABOVE: return sigm((ez - az) / p.tau_v);
    case FARM_BELOW: return sigm((az - ez) / p.tau_v);
    case FARM_NEAR: {
        const float dx = ex - ax, dy = ey - ay, dz = ez - az;
        const float d2 = dx * dx + dy * dy + dz * dz;
        return expf(-d2 / (2.f * p.sigma_near * p.sigma_near));
    }
    case FARM_LEFT_OF: return viewpoint_lr(ve, n_views, ex, ey, ez, ax, ay, az, 1.f, p);
    case FARM_RIGHT_OF: return viewpoint_lr(ve, n_views, ex, ey, ez, ax, ay, az, -1.f, p);
    default: return 0.f;
    }
}

__global__ void __launch_bounds__(TH)
compose_kernel(ComposeArgs a)
{
    __shared__ int32_t lm_idx[FARM_MAX_CONSTRAINTS][kMaxAnchorCands];
    __shared__ float lm_pos[FARM_MAX_CONSTRAINTS][kMaxAnchorCands][3];
    __shared__ int32_t cand_e[kMaxTargetCands];
    __shared__ float ssem[kMaxTargetCands];
    __shared__ uint16_t surv[kMaxTargetCands];
    __shared__ unsigned long long best[kMaxTargetCands][FARM_MAX_CONSTRAINTS];
    __shared__ uint64_t key[kMaxTargetCands];
    __shared__ uint16_t slot[kMaxTargetCands];
    __shared__ float s_thr;
    __shared__ int s_ns;

    const int64_t q = blockIdx.x;
    const int tid = threadIdx.x;
    const int32_t *meta = a.qmeta + q * 8;
    const int scene = meta[QM_SCENE];
    const int c_t = meta[QM_CLS];
    const int m = meta[QM_M];
    const int64_t c0 = meta[QM_C0];
    const int preds[4] = {meta[QM_PRED01] & 0xffff, (meta[QM_PRED01] >> 16) & 0xffff,
                          meta[QM_PRED23] & 0xffff, (meta[QM_PRED23] >> 16) & 0xffff};
    const int R = meta[QM_R];
    const int klm = meta[QM_KLM];
    const SceneDev sd = a.scenes[scene];
    const farm_params p = a.p;

    for (int t = tid; t < m * klm; t += TH) {
        const int i = t / klm, l = t - i * klm;
        const int32_t ai = a.lsel_idx[(c0 + i) * a.stride_l + l];
        lm_idx[i][l] = ai;
        lm_pos[i][l][0] = sd.pos[ai];
        lm_pos[i][l][1] = sd.pos[sd.n + ai];
        lm_pos[i][l][2] = sd.pos[2 * sd.n + ai];
    }
    const int32_t *cand = a.tsel_idx + q * a.stride_t;
    for (int c = tid; c < R; c += TH) {
        const int32_t e = cand[c];
        cand_e[c] = e;
        const float cf = (c_t >= 0 && sd.cls[e] != c_t) ? p.class_mis : 1.f;
        ssem[c] = cf / (p.mu + (float)(c + 1));
    }
    if (tid == 0) { s_thr = 0.f; s_ns = 0; }
    __syncthreads();
    // S_K = the k_max-th largest s_sem; candidates below (1 - w) S_K cannot
    // reach the TopK (k_max candidates score at least (1 - w) S_K).
    if (R > p.k_max) {
        for (int c = tid; c < R; c += TH) {
            const float v = ssem[c];
            int gt = 0, ge = 0;
            for (int j = 0; j < R; ++j) {
                gt += ssem[j] > v;
                ge += ssem[j] >= v;
            }
            if (gt < p.k_max && p.k_max <= ge) s_thr = (1.f - p.w) * v;
        }
    }
    __syncthreads();
    const float thr = s_thr;
    for (int c = tid; c < R; c += TH) {
        if (ssem[c] >= thr) {
            const int pos = atomicAdd(&s_ns, 1);
            surv[pos] = (uint16_t)c;
        }
    }
    __syncthreads();
    const int ns = s_ns;
    for (int t = tid; t < ns * FARM_MAX_CONSTRAINTS; t += TH) best[t / FARM_MAX_CONSTRAINTS][t % FARM_MAX_CONSTRAINTS] = 0ull;
    __syncthreads();
    // best witness per (survivor, constraint): max r, lower landmark index on ties
    const int per = m * klm;
    for (int t = tid; t < ns * per; t += TH) {
        const int pos = t / per;
        const int rem = t - pos * per;
        const int i = rem / klm, l = rem - i * klm;
        const int32_t e = cand_e[surv[pos]];
        const int32_t ai = lm_idx[i][l];
        if (ai == e) continue;
        const float ex = sd.pos[e], ey = sd.pos[sd.n + e], ez = sd.pos[2 * sd.n + e];
        const float *ve = sd.views + (int64_t)e * sd.n_views * kViewStride;
        const float r = relation(preds[i], ex, ey, ez, lm_pos[i][l][0], lm_pos[i][l][1], lm_pos[i][l][2], ve,
                                 sd.n_views, p);
        const unsigned long long k = ((unsigned long long)__float_as_uint(r) << 32) |
                                     (unsigned long long)(0xffffffffu - (uint32_t)ai);
        atomicMax(&best[pos][i], k);
    }
    __syncthreads();
    for (int pos = tid; pos < ns; pos += TH) {
        const int c = surv[pos];
        float t[FARM_MAX_CONSTRAINTS];
        bool zero = false;
        for (int i = 0; i < m; ++i) {
            const unsigned long long b = best[pos][i];
            t[i] = b ? __uint_as_float((uint32_t)(b >> 32)) : 0.f;
            zero |= !(t[i] > 0.f);
        }
        float g;
        if (m == 0) g = 1.f;
        else if (zero) g = 0.f;
        else if (m == 1) g = t[0];
        else if (m == 2) g = sqrtf(t[0] * t[1]);
        else if (m == 3) g = cbrtf(t[0] * t[1] * t[2]);
        else g = sqrtf(sqrtf(t[0] * t[1]) * sqrtf(t[2] * t[3]));
        const float s = ssem[c] * ((1.f - p.w) + p.w * g);
        key[pos] = ((uint64_t)order_key(s) << 32) | (uint64_t)(0xffffffffu - (uint32_t)cand_e[c]);
        slot[pos] = (uint16_t)pos;
    }
    int P = 1;
    while (P < ns) P <<= 1;
    for (int c = ns + tid; c < P; c += TH) { key[c] = 0ull; slot[c] = 0; }
    __syncthreads();
    for (int k = 2; k <= P; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = tid; i < P; i += TH) {
                const int ixj = i ^ j;
                if (ixj > i) {
                    const uint64_t x = key[i], y = key[ixj];
                    const bool desc = (i & k) == 0;
                    if (desc ? (x < y) : (x > y)) {
                        key[i] = y; key[ixj] = x;
                        const uint16_t u = slot[i]; slot[i] = slot[ixj]; slot[ixj] = u;
                    }
                }
            }
            __syncthreads();
        }
    }
    const int64_t ob = q * a.stride_t;
    for (int c = tid; c < a.stride_t; c += TH) {
        if (c < ns) {
            const int pos = slot[c];
            const uint32_t kk = (uint32_t)(key[c] >> 32);
            const uint32_t u = (kk & 0x80000000u) ? (kk & 0x7fffffffu) : ~kk;
            a.out_idx[ob + c] = cand_e[surv[pos]];
            a.out_score[ob + c] = __uint_as_float(u);
            for (int i = 0; i < FARM_MAX_CONSTRAINTS; ++i) {
                const unsigned long long b = i < m ? best[pos][i] : 0ull;
                a.out_t[(ob + c) * 4 + i] = i < m ? (b ? __uint_as_float((uint32_t)(b >> 32)) : 0.f) : -1.f;
                a.out_anchor[(ob + c) * 4 + i] = (i < m && b) ? (int32_t)(0xffffffffu - (uint32_t)(b & 0xffffffffu)) : -1;
            }
        } else {
            a.out_idx[ob + c] = -1;
            a.out_score[ob + c] = 0.f;
            for (int i = 0; i < FARM_MAX_CONSTRAINTS; ++i) {
                a.out_t[(ob + c) * 4 + i] = -1.f;
                a.out_anchor[(ob + c) * 4 + i] = -1;
            }
        }
    }
}

__global__ void gather_topk_kernel(int64_t n_q, int32_t k, int32_t ld, const int32_t *__restrict__ perm,
                                   const int32_t *__restrict__ idx, const float *__restrict__ score,
                                   const float *__restrict__ t, const int32_t *__restrict__ anchor,
                                   int32_t *o_idx, float *o_score, float *o_t, int32_t *o_anchor)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_q * k) return;
    const int64_t qo = i / k;              // output (caller's) query
    const int32_t j = (int32_t)(i - qo * k);
    const int64_t qp = perm ? perm[qo] : qo;   // planned position of that query
    const int64_t src = qp * ld + j;
    o_idx[i] = idx[src];
    o_score[i] = score[src];
    if (o_t)
        for (int c = 0; c < 4; ++c) o_t[i * 4 + c] = t[src * 4 + c];
    if (o_anchor)
        for (int c = 0; c < 4; ++c) o_anchor[i * 4 + c] = anchor[src * 4 + c];
}

}  // namespace

cudaError_t launch_compose(const ComposeArgs &a, cudaStream_t s)
{
    if (a.n_q <= 0) return cudaSuccess;
    compose_kernel<<<(unsigned)a.n_q, TH, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_gather_topk(int64_t n_q, int32_t k, int32_t ld, const int32_t *perm,
                               const int32_t *idx, const float *score, const float *t,
                               const int32_t *anchor, int32_t *o_idx, float *o_score, float *o_t,
                               int32_t *o_anchor, cudaStream_t s)
{
    const int64_t total = n_q * k;
    if (total <= 0) return cudaSuccess;
    const int th = 256;
    gather_topk_kernel<<<(unsigned)((total + th - 1) / th), th, 0, s>>>(
        n_q, k, ld, perm, idx, score, t, anchor, o_idx, o_score, o_t, o_anchor);
    return cudaGetLastError();
}

}  // namespace farm
