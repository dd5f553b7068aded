// k_compose.cu -- relation evaluation, best-witness binding and composite
// scoring of every kept target candidate (App. D.2 steps 4-5; App. B).
//
// One CTA of 128 threads per query; shared memory is sized by the batch's longest lists.
// The query's landmark candidates (K_a per constraint, in rank order) and
// their centres are staged in shared memory.  For every
// kept target candidate of rank r the CTA computes
//   s_sem = cf / (mu + r)                       (cf = class_mis on a class mismatch)
// (cf * F, F the fused score of several channels, for fused batches)
// and the k_max-th largest s_sem, S_K.  k_max candidates score at least
// (1 - w) S_K, so a candidate with s_sem < (1 - w) S_K cannot enter any TopK of
// size <= k_max (its composite is at most s_sem); only the others are scored:
//   t_i   = max_{a in L_i, a != e} r_rho_i(e, a)   (bound anchor = argmax, lower index on ties)
//   gbar  = (prod_i t_i)^(1/m),  s = s_sem * ((1 - w) + w * gbar)
// one constraint at a time, the lanes of a warp taking consecutive (scored
// candidate, landmark) pairs so that a warp evaluates one predicate; the best
// witness of a candidate is the max over (r, ~index) of its pairs (a
// segmented shuffle reduction, or 64-bit shared-memory atomics).  Because the
// composite is non-decreasing in every t_i and the anchors only meet at the
// target, the best binding takes each anchor's best witness on its own (the
// star decomposition of App. B).  The CTA then orders the scored candidates by
// (s descending, object index ascending), each one's position counted against
// the others, and writes the first k_max, so that any TopK is a prefix.
#include "farm_internal.h"

namespace farm {
namespace {

constexpr int TH = 128;      // small CTAs: more queries resident per SM to hide the dependent loads

// 1 / (1 + e^-x) for x >= 0, e^x / (1 + e^x) below (no overflow, no
// cancellation), without a branch: the lanes of a warp hold arguments of
// either sign.
__device__ __forceinline__ float sigm(float x)
{
    const float e = expf(-fabsf(x));
    return (x >= 0.f ? 1.f : e) / (1.f + e);
}

__device__ __forceinline__ uint32_t order_key(float f)
{
    const uint32_t u = __float_as_uint(f + 0.0f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

// The relations' scale parameters as factors (a multiplication where the
// definition divides by a constant), computed once per CTA.
struct RelK {
    float inv_tau_v, inv_tau_h, inv_tau_d, inv_on_gate;
    float near_k, next_k, on_k;      // -1 / (2 sigma^2) of Near, NextTo, On's band
    float z_min;
};

__device__ __forceinline__ RelK rel_k(const farm_params &p)
{
    RelK k;
    k.inv_tau_v = 1.f / p.tau_v;
    k.inv_tau_h = 1.f / p.tau_h;
    k.inv_tau_d = 1.f / p.tau_d;
    k.inv_on_gate = 1.f / p.on_gate;
    k.near_k = -1.f / (2.f * p.sigma_near * p.sigma_near);
    k.next_k = -1.f / (2.f * p.sigma_next * p.sigma_next);
    k.on_k = -1.f / (2.f * p.on_band * p.on_band);
    k.z_min = p.z_min;
    return k;
}

// The candidate's stored views ve, kViewStride floats each: {ox, oy, oz, fx},
// {fy, fz, rx, ry} (origin, unit forward, unit right in the ground plane),
// {Ze, ue, 0, 0} (the candidate's own depth and image coordinate there,
// computed at upload).  Mean over the views in which both the candidate and
// the landmark at (ax, ay, az) lie deeper than z_min of
//   LR: sig(sign (u_a - u_e) / tau_h)  (sign +1 LeftOf, -1 RightOf)
//   depth: sig(sign (Z_a - Z_e) / tau_d)  (sign +1 InFrontOf, -1 Behind)
// and 0.5 when there is no such view.
template <bool LR>
__device__ float viewpoint(const float *__restrict__ ve, int n_views, float ax, float ay, float az, float sign,
                           const RelK &k)
{
    // (every view evaluated and the ones not counted masked out, so that the
    // lanes of a warp, which hold different landmarks, do not diverge)
    float acc = 0.f;
    int counted = 0;
#pragma unroll 2
    for (int v = 0; v < n_views; ++v) {
        const float *r = ve + v * kViewStride;
        const float2 zu = __ldg(reinterpret_cast<const float2 *>(r + 8));
        const float4 o = __ldg(reinterpret_cast<const float4 *>(r));        // ox, oy, oz, fx
        const float4 f = __ldg(reinterpret_cast<const float4 *>(r + 4));    // fy, fz, rx, ry
        const float dax = ax - o.x, day = ay - o.y, daz = az - o.z;
        const float Za = dax * o.w + day * f.x + daz * f.y;
        const bool ok = zu.x > k.z_min && Za > k.z_min;
        float sv;
        if (LR) {
            const float ua = (dax * f.z + day * f.w) / Za;
            sv = sigm(sign * (ua - zu.y) * k.inv_tau_h);
        } else {
            sv = sigm(sign * (Za - zu.x) * k.inv_tau_d);
        }
        acc += ok ? sv : 0.f;
        counted += ok ? 1 : 0;
    }
    return counted ? acc / (float)counted : 0.5f;
}

// s + e = a + b exactly (Knuth's TwoSum; round-to-nearest FP32, no
// reassociation: nvcc keeps IEEE semantics without fast-math).
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = a + b;
    const float bp = s - a, ap = s - bp;
    e = (a - ap) + (b - bp);
}

// a b - c d with an error of a few units in the last place of the result
// (Kahan's algorithm: the rounding error of c d recovered by an FMA).
__device__ __forceinline__ float diff_of_products(float a, float b, float c, float d)
{
    const float w = c * d;
    const float e = fmaf(-c, d, w);
    const float f = fmaf(a, b, -w);
    return f + e;
}

// Between(e, a_p, a_q): e's centre on the segment from a_p to a_q, t its
// projected position (0 at a_p, 1 at a_q) and d2 its squared distance from
// the line: sig(t / 0.1) sig((1 - t) / 0.1) exp(-d2 / (2 sigma_near^2)); 0 for
// coincident landmarks.
__device__ __forceinline__ float between_rel(float ex, float ey, float ez, const float *pp, const float *pq,
                                             const RelK &k)
{
    // rel = e - a_p and seg = a_q - a_p exactly, each as a rounded part plus
    // its error (TwoSum): the landmarks of a Between may lie a hundred metres
    // apart while e stays close to their line, and the rounding of those
    // differences would otherwise dominate d^2
    const float pe[3] = {ex, ey, ez};
    float rh[3], rl[3], sh[3], sl[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        two_sum(pe[k], -pp[k], rh[k], rl[k]);
        two_sum(pq[k], -pp[k], sh[k], sl[k]);
    }
    const float ss = sh[0] * sh[0] + sh[1] * sh[1] + sh[2] * sh[2];
    if (!(ss > 0.f)) return 0.f;
    const float t = (rh[0] * sh[0] + rh[1] * sh[1] + rh[2] * sh[2]) / ss;
    // d^2 = |rel x seg|^2 / |seg|^2 (free of t's rounding); each component
    // a b - c d by Kahan's FMA difference of products, plus the first-order
    // terms of the low parts
    float c[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const int i = (k + 1) % 3, j = (k + 2) % 3;
        c[k] = diff_of_products(rh[i], sh[j], rh[j], sh[i]) +
               ((rh[i] * sl[j] + rl[i] * sh[j]) - (rh[j] * sl[i] + rl[j] * sh[i]));
    }
    const float d2 = (c[0] * c[0] + c[1] * c[1] + c[2] * c[2]) / ss;
    return sigm(t / 0.1f) * sigm((1.f - t) / 0.1f) * expf(d2 * k.near_k);
}

// What a relation needs beyond the two objects: the candidate's stored views
// and the query's Closest / Farthest candidate set (its kc best target
// candidates, indices and centres).
struct RelCtx {
    const float *ve;           // the candidate's views [n_views][kViewStride] (global)
    int n_views;
    const int32_t *cset_idx;
    const float *cset_pos;     // [kc][3]
    int kc;
};

// r_rho(e, a) (App. D.2 step 4).  ce: e's position in the query's target
// list (rank - 1), which decides membership of the Closest / Farthest set.
__device__ __forceinline__ float relation(int pred, int32_t e, int ce, float ex, float ey, float ez, float esx,
                                          float esy, float esz, int32_t ai, float ax, float ay, float az, float asx,
                                          float asy, float asz, const RelCtx &rc, const RelK &k)
{
    switch (pred) {
    case FARM_NEAR_H: {
        // 1 - H with box-moment Gaussians (variance s^2 / 12 per axis):
        // ln BC = sum_k 0.5 log(1 - (|s_e| - |s_a|)^2 / q) - 3 d^2 / q,
        // q = s_e^2 + s_a^2, and H^2 = 1 - BC = -expm1(ln BC), which keeps
        // its relative accuracy when the two Gaussians nearly coincide
        const float se[3] = {fabsf(esx), fabsf(esy), fabsf(esz)}, sa[3] = {fabsf(asx), fabsf(asy), fabsf(asz)};
        const float d[3] = {ex - ax, ey - ay, ez - az};
        float lbc = 0.f;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const float q = se[k] * se[k] + sa[k] * sa[k];
            if (q == 0.f) {
                if (d[k] != 0.f) return 0.f;      // two flat boxes at different levels
                continue;
            }
            const float dd = se[k] - sa[k];
            lbc += 0.5f * log1pf(-(dd * dd) / q) - 3.f * d[k] * d[k] / q;
        }
        // 1 - H = BC / (1 + H): no cancellation when BC is small either, where
        // the geometric mean of App. D.2 step 5 would magnify a relative error
        return expf(lbc) / (1.f + sqrtf(fmaxf(-expm1f(lbc), 0.f)));
    }
    case FARM_INSIDE: {
        // the fraction of e's box inside a's box.  Per axis the overlap is
        // 2 h_e, 2 h_a, or h_e + h_a -/+ (a - e) (h the half sizes); the last
        // two are summed without rounding error until the final add (TwoSum),
        // so that a thin overlap keeps its relative accuracy -- the geometric
        // mean of App. D.2 step 5 magnifies the relative error of a small score
        const float pe[3] = {ex, ey, ez}, pa[3] = {ax, ay, az};
        const float he[3] = {0.5f * fabsf(esx), 0.5f * fabsf(esy), 0.5f * fabsf(esz)};
        const float ha[3] = {0.5f * fabsf(asx), 0.5f * fabsf(asy), 0.5f * fabsf(asz)};
        float frac = 1.f;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            float d1, d2;                    // a - e = d1 + d2 exactly
            two_sum(pa[k], -pe[k], d1, d2);
            if (he[k] == 0.f) {
                if (!(fabsf(d1) <= ha[k])) return 0.f;
                continue;
            }
            const bool top_e = he[k] - ha[k] <= d1;       // e's upper face is the upper bound
            const bool bot_e = d1 <= ha[k] - he[k];       // e's lower face is the lower bound
            float ov;
            if (top_e && bot_e) {
                ov = 2.f * he[k];
            } else if (!top_e && !bot_e) {
                ov = 2.f * ha[k];
            } else {
                float t1, t2, u1, u2;
                two_sum(he[k], ha[k], t1, t2);            // h_e + h_a = t1 + t2
                const float sg = top_e ? -1.f : 1.f;      // top_e: h_e + h_a - (a - e); else + (a - e)
                two_sum(t1, sg * d1, u1, u2);
                ov = u1 + (u2 + (t2 + sg * d2));
                ov = fminf(ov, 2.f * fminf(he[k], ha[k]));
            }
            if (!(ov > 0.f)) return 0.f;
            frac *= ov / (2.f * he[k]);
        }
        return frac;
    }
    case FARM_ABOVE: return sigm((ez - az) * k.inv_tau_v);
    case FARM_BELOW: return sigm((az - ez) * k.inv_tau_v);
    case FARM_NEAR:
    case FARM_NEXT_TO: {
        const float dx = ex - ax, dy = ey - ay, dz = ez - az;
        const float d2 = dx * dx + dy * dy + dz * dz;
        return expf(d2 * (pred == FARM_NEAR ? k.near_k : k.next_k));
    }
    case FARM_ON: {
        const float dx = ex - ax, dy = ey - ay;
        const float rho = 0.5f * fmaxf(asx, asy);
        const float gate = sigm((rho - sqrtf(dx * dx + dy * dy)) * k.inv_on_gate);
        const float gap = (ez - 0.5f * esz) - (az + 0.5f * asz);
        return gate * expf(gap * gap * k.on_k);
    }
    case FARM_LEFT_OF: return viewpoint<true>(rc.ve, rc.n_views, ax, ay, az, 1.f, k);
    case FARM_RIGHT_OF: return viewpoint<true>(rc.ve, rc.n_views, ax, ay, az, -1.f, k);
    case FARM_IN_FRONT_OF: return viewpoint<false>(rc.ve, rc.n_views, ax, ay, az, 1.f, k);
    case FARM_BEHIND: return viewpoint<false>(rc.ve, rc.n_views, ax, ay, az, -1.f, k);
    case FARM_CLOSEST:
    case FARM_FARTHEST: {
        if (ce >= rc.kc) return 0.f;                // e is not in the candidate set
        const float dx = ex - ax, dy = ey - ay, dz = ez - az;
        const float de = dx * dx + dy * dy + dz * dz;
        int members = 0, closer = 0;
        for (int k = 0; k < rc.kc; ++k) {
            const int32_t j = rc.cset_idx[k];
            if (j == ai) continue;
            ++members;
            const float jx = rc.cset_pos[3 * k] - ax, jy = rc.cset_pos[3 * k + 1] - ay, jz = rc.cset_pos[3 * k + 2] - az;
            const float dj = jx * jx + jy * jy + jz * jz;
            closer += (dj < de || (dj == de && j < e)) ? 1 : 0;
        }
        const int rank = 1 + closer;
        return pred == FARM_CLOSEST ? 1.f / (float)rank : 1.f / (float)(members - rank + 1);
    }
    default: return 0.f;
    }
}

constexpr int WARPS = TH / 32;

// Shared-memory layout of one query, sized by the batch's longest target list
// RM, landmark list KM and Closest /
// Farthest set KC; every section starts on a 16-byte boundary.
struct ComposeSmem {
    size_t best, key, sv, lm, cset_pos, lm_idx, cand_e, ssem, surv, bytes;
    __host__ __device__ static size_t up16(size_t x) { return (x + 15) & ~(size_t)15; }
    __host__ __device__ ComposeSmem(int RM, int KM, int KC)
    {
        size_t o = 0;
        best = o;   o = up16(o + (size_t)RM * FARM_MAX_CONSTRAINTS * 8);
        key = o;    o = up16(o + (size_t)RM * 8);
        sv = o;     o = up16(o + (size_t)RM * 32);
        lm = o;     o = up16(o + (size_t)FARM_MAX_CONSTRAINTS * KM * 32);
        cset_pos = o; o = up16(o + (size_t)KC * 3 * 4);
        lm_idx = o; o = up16(o + (size_t)FARM_MAX_CONSTRAINTS * KM * 4);
        cand_e = o; o = up16(o + (size_t)RM * 4);
        ssem = o;   o = up16(o + (size_t)RM * 4);
        surv = o;   o = up16(o + (size_t)RM * 2);
        bytes = o;
    }
};

__global__ void __launch_bounds__(TH, 10)
compose_kernel(ComposeArgs a, int32_t KC)
{
    extern __shared__ __align__(16) uint8_t sm[];
    const int RM = a.stride_t, KM = a.stride_l;
    const ComposeSmem L(RM, KM, KC);
    unsigned long long *best = reinterpret_cast<unsigned long long *>(sm + L.best);   // [RM][4]
    uint64_t *key = reinterpret_cast<uint64_t *>(sm + L.key);
    // per survivor: {ex, ey, ez, esx}, {esy, esz, e, list position}
    float4 *sv = reinterpret_cast<float4 *>(sm + L.sv);                               // [RM][2]
    // per landmark: {ax, ay, az, asx}, {asy, asz, 0, 0}
    float4 *lm = reinterpret_cast<float4 *>(sm + L.lm);                               // [4][KM][2]
    float *cset_pos = reinterpret_cast<float *>(sm + L.cset_pos);                     // [KC][3]
    int32_t *lm_idx = reinterpret_cast<int32_t *>(sm + L.lm_idx);                     // [4][KM]
    int32_t *cand_e = reinterpret_cast<int32_t *>(sm + L.cand_e);
    float *ssem = reinterpret_cast<float *>(sm + L.ssem);
    uint16_t *surv = reinterpret_cast<uint16_t *>(sm + L.surv);
    __shared__ float s_thr;
    __shared__ int s_ns;

    const int64_t q = blockIdx.x;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int32_t *meta = a.qmeta + q * 8;
    const int scene = meta[QM_SCENE];
    const int c_t = meta[QM_CLS];
    const int m = meta[QM_M];
    const int64_t c0 = meta[QM_C0];
    // the four predicate codes (each < 256) packed a byte apiece, so that a
    // lane indexes them without a local-memory array
    const uint32_t predw = (uint32_t)(meta[QM_PRED01] & 0xff) | (uint32_t)((meta[QM_PRED01] >> 16) & 0xff) << 8 |
                           (uint32_t)(meta[QM_PRED23] & 0xff) << 16 | (uint32_t)((meta[QM_PRED23] >> 16) & 0xff) << 24;
    auto pred_of = [predw](int i) { return (int)((predw >> (8 * i)) & 0xffu); };
    const int R = meta[QM_R];
    const int klm = meta[QM_KLM];
    const SceneDev sd = a.scenes[scene];
    const farm_params p = a.p;
    const int kc = min(min(p.k_closest, R), KC);     // the Closest / Farthest set: target ranks 1..kc

    const RelK K = rel_k(p);

    // (an index outside the scene never reaches a memory access: such a
    // landmark is skipped and such a candidate never survives)
    const int32_t *cand = a.tsel_idx + q * a.stride_t;
    for (int c = tid; c < R; c += TH) {
        const int32_t e = cand[c];
        const bool ok = e >= 0 && e < sd.n;
        cand_e[c] = ok ? e : -1;
        const float cf = (c_t >= 0 && ok && sd.cls[e] != c_t) ? p.class_mis : 1.f;
        ssem[c] = ok ? (a.tsel_F ? cf * a.tsel_F[q * a.stride_t + c] : cf / (p.mu + (float)(c + 1))) : -1.f;
        if (c < kc) {
            cset_pos[3 * c + 0] = ok ? sd.pos[e] : 0.f;
            cset_pos[3 * c + 1] = ok ? sd.pos[sd.n + e] : 0.f;
            cset_pos[3 * c + 2] = ok ? sd.pos[2 * sd.n + e] : 0.f;
        }
    }
    for (int x = tid; x < R * FARM_MAX_CONSTRAINTS; x += TH) best[x] = 0ull;
    if (tid == 0) { s_thr = 0.f; s_ns = 0; }
    __syncthreads();
    // the landmark lists; S_K = the k_max-th largest s_sem (each candidate's
    // rank counted against the others): candidates below (1 - w) S_K cannot
    // reach the TopK (k_max candidates score at least (1 - w) S_K)
    for (int t = tid; t < m * klm; t += TH) {
        const int i = t / klm, l = t - i * klm;
        int32_t ai = a.lsel_idx[(c0 + i) * a.stride_l + l];
        if (ai < 0 || ai >= sd.n) ai = -1;
        lm_idx[i * KM + l] = ai;
        lm[2 * (i * KM + l)] = ai >= 0 ? make_float4(sd.pos[ai], sd.pos[sd.n + ai], sd.pos[2 * sd.n + ai], sd.size[ai])
                                       : make_float4(0.f, 0.f, 0.f, 0.f);
        lm[2 * (i * KM + l) + 1] = ai >= 0 ? make_float4(sd.size[sd.n + ai], sd.size[2 * sd.n + ai], 0.f, 0.f)
                                           : make_float4(0.f, 0.f, 0.f, 0.f);
    }
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
        const int32_t e = cand_e[c];
        if (ssem[c] >= thr && e >= 0) {
            const int pos = atomicAdd(&s_ns, 1);
            surv[pos] = (uint16_t)c;
            sv[2 * pos] = make_float4(__ldg(sd.pos + e), __ldg(sd.pos + sd.n + e), __ldg(sd.pos + 2 * sd.n + e),
                                      __ldg(sd.size + e));
            sv[2 * pos + 1] = make_float4(__ldg(sd.size + sd.n + e), __ldg(sd.size + 2 * sd.n + e),
                                          __int_as_float(e), __int_as_float(c));
        }
    }
    __syncthreads();
    const int ns = s_ns;
    // best witness per (survivor, constraint): for one constraint at a time
    // (so that a warp evaluates one predicate and its lanes do not diverge on
    // it) the lanes take consecutive (survivor, landmark) pairs; the best
    // (r, ~index) of a survivor -- the largest r, then the lower landmark
    // index -- is the max over its pairs: a shuffle reduction over aligned
    // groups of klm lanes when klm is a power of two up to 32, else 64-bit
    // shared-memory atomics.  r >= 0, so its bits order like the float, and a
    // zero word means no witness.
    const bool pow2 = klm <= 32 && (klm & (klm - 1)) == 0;
    const int lk = pow2 ? __ffs(klm) - 1 : 0;
    const int pairs = ns * klm;
    for (int i = 0; i < m; ++i) {
        const int pr = pred_of(i);
        if (pr >= FARM_BETWEEN) continue;        // Between pairs: below
        for (int base = warp * 32; base < pairs; base += TH) {
            const int t = base + lane;
            int sidx = 0;
            uint32_t h = 0u, lo = 0u;
            if (t < pairs) {
                sidx = pow2 ? t >> lk : t / klm;
                const int l = t - sidx * klm;
                const float4 sa = sv[2 * sidx], sb = sv[2 * sidx + 1];
                const int32_t e = __float_as_int(sb.z);
                const int ce = __float_as_int(sb.w);
                const int32_t ai = lm_idx[i * KM + l];
                if (ai >= 0 && ai != e) {
                    const float ex = sa.x, ey = sa.y, ez = sa.z, esx = sa.w, esy = sb.x, esz = sb.y;
                    const float4 la = lm[2 * (i * KM + l)], lb = lm[2 * (i * KM + l) + 1];
                    const RelCtx rc{sd.views + (int64_t)e * sd.n_views * kViewStride, sd.n_views, cand_e, cset_pos, kc};
                    const float r = relation(pr, e, ce, ex, ey, ez, esx, esy, esz, ai, la.x, la.y, la.z, la.w, lb.x,
                                             lb.y, rc, K);
                    h = __float_as_uint(r);
                    lo = 0xffffffffu - (uint32_t)ai;
                }
            }
            if (pow2) {
                for (int off = klm >> 1; off > 0; off >>= 1) {
                    const uint32_t oh = __shfl_xor_sync(0xffffffffu, h, off);
                    const uint32_t ol = __shfl_xor_sync(0xffffffffu, lo, off);
                    if (oh > h || (oh == h && ol > lo)) { h = oh; lo = ol; }
                }
                if (t < pairs && (lane & (klm - 1)) == 0)
                    best[sidx * FARM_MAX_CONSTRAINTS + i] = ((unsigned long long)h << 32) | lo;
            } else if (h | lo) {
                atomicMax(&best[sidx * FARM_MAX_CONSTRAINTS + i], ((unsigned long long)h << 32) | lo);
            }
        }
    }
    // Between pairs (constraints c, c + 1): the best (a_p, a_q) over
    // L_c x L_{c+1} -- exact elimination of the pair -- with the larger r,
    // then the lower a_p, then the lower a_q; one warp per survivor
    bool any_between = false;
    for (int c = 0; c + 1 < m; ++c) any_between |= pred_of(c) == FARM_BETWEEN;
    if (any_between) {
        for (int pos = warp; pos < ns; pos += WARPS) {
            const float4 sa = sv[2 * pos];
            const int32_t e = __float_as_int(sv[2 * pos + 1].z);
            const float ex = sa.x, ey = sa.y, ez = sa.z;
            for (int c = 0; c + 1 < m; ++c) {
                if (pred_of(c) != FARM_BETWEEN) continue;
                uint32_t h = 0u, wp = 0u, wq = 0u;
                for (int t = lane; t < klm * klm; t += 32) {
                    const int x = t / klm, y = t - x * klm;
                    const int32_t ap = lm_idx[c * KM + x], aq = lm_idx[(c + 1) * KM + y];
                    if (ap < 0 || aq < 0 || ap == e || aq == e || ap == aq) continue;
                    const float r = between_rel(ex, ey, ez, reinterpret_cast<const float *>(lm + 2 * (c * KM + x)),
                                                reinterpret_cast<const float *>(lm + 2 * ((c + 1) * KM + y)), K);
                    const uint32_t rh = __float_as_uint(r), lp = 0xffffffffu - (uint32_t)ap,
                                   lq = 0xffffffffu - (uint32_t)aq;
                    if (rh > h || (rh == h && (lp > wp || (lp == wp && lq > wq)))) { h = rh; wp = lp; wq = lq; }
                }
                const uint32_t hm = __reduce_max_sync(0xffffffffu, h);
                const uint32_t pm = __reduce_max_sync(0xffffffffu, h == hm ? wp : 0u);
                const uint32_t qm = __reduce_max_sync(0xffffffffu, (h == hm && wp == pm) ? wq : 0u);
                if (lane == 0) {
                    best[pos * FARM_MAX_CONSTRAINTS + c] = ((unsigned long long)hm << 32) | pm;
                    best[pos * FARM_MAX_CONSTRAINTS + c + 1] = ((unsigned long long)hm << 32) | qm;
                }
            }
        }
    }
    __syncthreads();
    for (int pos = tid; pos < ns; pos += TH) {
        const int c = surv[pos];
        // the factors of the geometric mean: a Between pair counts once
        float t[FARM_MAX_CONSTRAINTS];
        int mf = 0;
        bool zero = false;
        for (int i = 0; i < m; ++i) {
            if (pred_of(i) == FARM_BETWEEN_AND) continue;
            const unsigned long long b = best[pos * FARM_MAX_CONSTRAINTS + i];
            t[mf] = b ? __uint_as_float((uint32_t)(b >> 32)) : 0.f;
            zero |= !(t[mf] > 0.f);
            ++mf;
        }
        float g;
        if (mf == 0) g = 1.f;
        else if (zero) g = 0.f;
        else if (mf == 1) g = t[0];
        else if (mf == 2) g = sqrtf(t[0] * t[1]);
        else if (mf == 3) g = cbrtf(t[0] * t[1] * t[2]);
        else g = sqrtf(sqrtf(t[0] * t[1]) * sqrtf(t[2] * t[3]));
        const float s = ssem[c] * ((1.f - p.w) + p.w * g);
        key[pos] = ((uint64_t)order_key(s) << 32) | (uint64_t)(0xffffffffu - (uint32_t)cand_e[c]);
    }
    __syncthreads();
    // the scored candidates in (s desc, object index asc) order are the key
    // order, all keys distinct: each one's position is the number of larger
    // keys; only a TopK prefix of at most k_max entries is ever read
    const int64_t ob = q * a.stride_t;
    const int n_out = min(a.stride_t, max(p.k_max, 1));
    for (int pos = tid; pos < ns; pos += TH) {
        const uint64_t kp = key[pos];
        int c = 0;
        for (int j = 0; j < ns; ++j) c += key[j] > kp ? 1 : 0;
        if (c >= n_out) continue;
        const uint32_t kk = (uint32_t)(kp >> 32);
        const uint32_t u = (kk & 0x80000000u) ? (kk & 0x7fffffffu) : ~kk;
        a.out_idx[ob + c] = cand_e[surv[pos]];
        a.out_score[ob + c] = __uint_as_float(u);
        for (int i = 0; i < FARM_MAX_CONSTRAINTS; ++i) {
            const unsigned long long b = i < m ? best[pos * FARM_MAX_CONSTRAINTS + i] : 0ull;
            a.out_t[(ob + c) * 4 + i] = i < m ? (b ? __uint_as_float((uint32_t)(b >> 32)) : 0.f) : -1.f;
            a.out_anchor[(ob + c) * 4 + i] = (i < m && b) ? (int32_t)(0xffffffffu - (uint32_t)(b & 0xffffffffu)) : -1;
        }
    }
    for (int c = ns + tid; c < n_out; c += TH) {
        a.out_idx[ob + c] = -1;
        a.out_score[ob + c] = 0.f;
        for (int i = 0; i < FARM_MAX_CONSTRAINTS; ++i) {
            a.out_t[(ob + c) * 4 + i] = -1.f;
            a.out_anchor[(ob + c) * 4 + i] = -1;
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
    if (a.stride_t < 1 || a.stride_t > kMaxTargetCands || a.stride_l < 1 || a.stride_l > kMaxAnchorCands)
        return cudaErrorInvalidValue;
    const int KC = a.p.k_closest < a.stride_t ? a.p.k_closest : a.stride_t;
    const ComposeSmem L(a.stride_t, a.stride_l, KC);
    if (L.bytes + 64 > 48 * 1024) {     // (plus the kernel's few bytes of static shared memory)
        const cudaError_t e = cudaFuncSetAttribute(compose_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   (int)L.bytes);
        if (e != cudaSuccess) return e;
    }
    compose_kernel<<<(unsigned)a.n_q, TH, L.bytes, s>>>(a, KC);
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
