// k_assoc.cu -- mapping-side association of a batch of detections with the
// memory's entities (App. D.1 steps 3-5), each a 3D Gaussian (mean;
// covariance packed xx, xy, xz, yy, yz, zz) with an appearance feature:
//
//  * neighbour search: from the detection-by-entity feature cosines (the
//    FP32-accurate similarity kernel), the active entities with cosine >=
//    tau_f get the Hellinger distance
//      H = sqrt(1 - BC),  ln BC = (ln det S_d + ln det S_e) / 4 - ln det S / 2
//                                 - dmu' S^-1 dmu / 8,  S = (S_d + S_e) / 2,
//    (1 - BC evaluated as -expm1(ln BC)); those with H <= h_max are sorted by
//    (H, index) and the first max_m kept (one CTA per detection);
//  * correspondence: the connected components of the graph joining each
//    detection (node N + d) to its matches, by min-label hooking and pointer
//    jumping (one CTA: the graph has at most B x max_m edges); the winner of a
//    component is its entity of largest weight (lower index on ties), a
//    component without an entity is a lone detection that starts a new
//    entity;
//  * fusion: every slot adds w (mu - c) and w f into its winner (c the
//    winner's own mean: a shift that keeps FP32 digits at site coordinates),
//    then w (S + (mu - mu_g)(mu - mu_g)') -- the sufficient-statistics merge
//    M1 = w mu, M2 = w (S + mu mu') in a form free of the cancellation of
//    M2 / w - mu mu'.  Sums use atomics, so their order (and the last bits)
//    may vary from run to run.
#include "farm_internal.h"

namespace farm {
namespace {

constexpr int TA = 128;
constexpr int CAPA = 1024;       // candidates within the budget a detection may have
constexpr int CAPP = 4096;       // prefilter list: entities past the cosine threshold awaiting evaluation
constexpr int PER_PASS = TA * 16;   // entries one streaming pass can add (four float4 per thread)

__device__ __forceinline__ float det3f(const float c[6])
{
    return c[0] * (c[3] * c[5] - c[4] * c[4]) - c[1] * (c[1] * c[5] - c[4] * c[2]) +
           c[2] * (c[1] * c[4] - c[3] * c[2]);
}

// Hellinger distance of two Gaussians; 1 for a degenerate covariance.
__device__ float hellinger_f(const float m1[3], const float c1[6], const float m2[3], const float c2[6])
{
    float S[6], d[3];
#pragma unroll
    for (int k = 0; k < 6; ++k) S[k] = 0.5f * (c1[k] + c2[k]);
#pragma unroll
    for (int k = 0; k < 3; ++k) d[k] = m1[k] - m2[k];
    const float dS = det3f(S), d1 = det3f(c1), d2 = det3f(c2);
    if (!(dS > 0.f) || !(d1 > 0.f) || !(d2 > 0.f)) return 1.f;
    const float a0 = S[3] * S[5] - S[4] * S[4], a1 = S[2] * S[4] - S[1] * S[5], a2 = S[1] * S[4] - S[2] * S[3];
    const float a3 = S[0] * S[5] - S[2] * S[2], a4 = S[1] * S[2] - S[0] * S[4], a5 = S[0] * S[3] - S[1] * S[1];
    const float x0 = a0 * d[0] + a1 * d[1] + a2 * d[2];
    const float x1 = a1 * d[0] + a3 * d[1] + a4 * d[2];
    const float x2 = a2 * d[0] + a4 * d[1] + a5 * d[2];
    const float q = (d[0] * x0 + d[1] * x1 + d[2] * x2) / dS;
    const float lbc = 0.25f * (logf(d1) + logf(d2)) - 0.5f * logf(dS) - 0.125f * q;
    return sqrtf(fmaxf(-expm1f(lbc), 0.f));
}

// The Hellinger distance of detection (md, cd) to entity e, -1 for an
// inactive entity.  Kept out of line: the streaming loop that calls it for
// the few entities past the cosine prefilter is unrolled sixteen-fold, and
// inlining it there overflowed the instruction cache.
__device__ __noinline__ float entity_distance(int e, int32_t N, const float *__restrict__ ent_mu,
                                              const float *__restrict__ ent_cov,
                                              const int32_t *__restrict__ ent_active, const float md[3],
                                              const float cd[6])
{
    if (!ent_active[e]) return -1.f;
    float me[3], ce[6];
#pragma unroll
    for (int k = 0; k < 3; ++k) me[k] = ent_mu[(int64_t)k * N + e];
#pragma unroll
    for (int k = 0; k < 6; ++k) ce[k] = ent_cov[(int64_t)k * N + e];
    return hellinger_f(md, cd, me, ce);
}

__global__ void __launch_bounds__(TA)
assoc_search_kernel(const float *__restrict__ S, int64_t ld, int32_t N, int32_t B, const float *__restrict__ ent_mu,
                    const float *__restrict__ ent_cov, const int32_t *__restrict__ ent_active,
                    const float *__restrict__ det_mu, const float *__restrict__ det_cov, float tau_f, float h_max,
                    int32_t max_m, int32_t *__restrict__ match_cnt, int32_t *__restrict__ match_idx,
                    float *__restrict__ match_h, int32_t *err)
{
    __shared__ uint64_t cand[CAPA];
    __shared__ int32_t pre[CAPP];
    __shared__ int s_cnt, s_np;
    const int d = blockIdx.x, tid = threadIdx.x;
    if (tid == 0) {
        s_cnt = 0;
        s_np = 0;
    }
    __syncthreads();
    float md[3], cd[6];
#pragma unroll
    for (int k = 0; k < 3; ++k) md[k] = det_mu[(int64_t)k * B + d];
#pragma unroll
    for (int k = 0; k < 6; ++k) cd[k] = det_cov[(int64_t)k * B + d];
    // the row is streamed in float4 loads, four in flight per thread (its
    // leading dimension is a multiple of 32 floats, so the row is 16-byte
    // aligned and a load never leaves it); the entities past the cosine
    // prefilter are listed in shared memory and evaluated by all threads
    // together (one entity per thread), whenever the list could overflow in
    // the next pass and at the end: evaluated where they are found, they
    // would each run on one lane of a warp
    const float *row = S + (int64_t)d * ld;
    const float4 *row4 = reinterpret_cast<const float4 *>(row);
    const int n4 = (N + 3) >> 2;
    auto evaluate = [&](int np) {
        for (int i = tid; i < np; i += TA) {
            const int e = pre[i];
            const float h = entity_distance(e, N, ent_mu, ent_cov, ent_active, md, cd);
            if (h >= 0.f && h <= h_max) {
                const int pos = atomicAdd(&s_cnt, 1);
                if (pos < CAPA) cand[pos] = ((uint64_t)__float_as_uint(h) << 32) | (uint32_t)e;   // H >= 0: bits order like H
            }
        }
    };
    for (int g0 = 0; g0 < n4; g0 += TA * 4) {
        float4 v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int g = g0 + u * TA + tid;
            v[u] = g < n4 ? __ldcs(row4 + g) : make_float4(-2.f, -2.f, -2.f, -2.f);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int e0 = 4 * (g0 + u * TA + tid);
            const float x[4] = {v[u].x, v[u].y, v[u].z, v[u].w};
#pragma unroll
            for (int c = 0; c < 4; ++c)
                if (x[c] >= tau_f && e0 + c < N) pre[atomicAdd(&s_np, 1)] = e0 + c;
        }
        __syncthreads();
        const int np = s_np;
        if (np > CAPP - PER_PASS) {      // (uniform) at most PER_PASS more could come in the next pass
            evaluate(np);
            __syncthreads();
            if (tid == 0) s_np = 0;
            __syncthreads();
        }
    }
    evaluate(s_np);
    __syncthreads();
    const int cnt = s_cnt;
    if (cnt > CAPA) {
        if (tid == 0) atomicOr(err, kErrAssocOverflow);
    }
    const int nc = min(cnt, CAPA);
    int P = 1;
    while (P < nc) P <<= 1;
    for (int i = nc + tid; i < P; i += TA) cand[i] = ~0ull;
    __syncthreads();
    for (int k = 2; k <= P; k <<= 1) {           // ascending: smaller H, then lower index, first
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = tid; i < P; i += TA) {
                const int ixj = i ^ j;
                if (ixj > i) {
                    const uint64_t a = cand[i], b = cand[ixj];
                    const bool up = (i & k) == 0;
                    if (up ? (a > b) : (a < b)) { cand[i] = b; cand[ixj] = a; }
                }
            }
            __syncthreads();
        }
    }
    if (tid == 0) match_cnt[d] = cnt;
    for (int j = tid; j < max_m; j += TA) {
        const bool has = j < nc;
        match_idx[(int64_t)d * max_m + j] = has ? (int32_t)(cand[j] & 0xffffffffu) : -1;
        match_h[(int64_t)d * max_m + j] = has ? __uint_as_float((uint32_t)(cand[j] >> 32)) : -1.f;
    }
}

// Connected components of the match graph: label[t] ends as the smallest
// node of t's component.  One CTA; hooking rounds until nothing changes (at
// most max_rounds, else the error bit).  With in_smem the labels live in
// shared memory (T * 4 bytes of dynamic shared memory) and are written to
// `label` at the end; otherwise they are worked on in `label` directly.
__global__ void __launch_bounds__(1024)
assoc_components_kernel(int32_t N, int32_t B, int32_t max_m, const int32_t *__restrict__ match_idx,
                        int32_t *label_out, int32_t max_rounds, int32_t *err, int32_t in_smem)
{
    extern __shared__ int32_t s_label[];
    __shared__ int s_changed;
    const int T = N + B, tid = threadIdx.x;
    int32_t *label = in_smem ? s_label : label_out;
    for (int t = tid; t < T; t += blockDim.x) label[t] = t;
    __syncthreads();
    const int E = B * max_m;
    int round = 0;
    for (; round < max_rounds; ++round) {
        if (tid == 0) s_changed = 0;
        __syncthreads();
        // hooking: the parent of the larger label takes the smaller one
        for (int k = tid; k < E; k += blockDim.x) {
            const int e = match_idx[k];
            if (e < 0) continue;
            const int u = N + k / max_m;
            const int pu = ((volatile int32_t *)label)[u], pv = ((volatile int32_t *)label)[e];
            if (pu != pv) {
                atomicMin(&label[max(pu, pv)], min(pu, pv));
                s_changed = 1;
            }
        }
        __syncthreads();
        // pointer jumping until every node points at a root
        for (int t = tid; t < T; t += blockDim.x) {
            int l = label[t];
            for (int it = 0; it < 4096; ++it) {
                const int ll = ((volatile int32_t *)label)[l];
                if (ll == l) break;
                l = ll;
            }
            label[t] = l;
        }
        __syncthreads();
        if (!s_changed) break;
        __syncthreads();
    }
    if (tid == 0 && round >= max_rounds) atomicOr(err, kErrTimeout);
    if (in_smem)
        for (int t = tid; t < T; t += blockDim.x) label_out[t] = s_label[t];
}

// win[r]: the heaviest entity of component r as (w bits, ~index).
__global__ void assoc_winner_kernel(int32_t N, const float *__restrict__ ent_w, const int32_t *__restrict__ label,
                                    unsigned long long *win)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= N) return;
    const unsigned long long k = ((unsigned long long)__float_as_uint(fmaxf(ent_w[e], 0.f)) << 32) |
                                 (unsigned long long)(0xffffffffu - (uint32_t)e);
    atomicMax(&win[label[e]], k);
}

__global__ void assoc_parent_kernel(int32_t T, const int32_t *__restrict__ label,
                                    const unsigned long long *__restrict__ win, int32_t *parent)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= T) return;
    const unsigned long long k = win[label[t]];
    parent[t] = k ? (int32_t)(0xffffffffu - (uint32_t)(k & 0xffffffffu)) : t;
}

struct Slots {
    int32_t N, B, F;
    const float *ent_mu, *ent_cov, *ent_feat, *ent_w, *det_mu, *det_cov, *det_feat;
    __device__ float mu(int t, int k) const { return t < N ? ent_mu[(int64_t)k * N + t] : det_mu[(int64_t)k * B + (t - N)]; }
    __device__ float cv(int t, int k) const { return t < N ? ent_cov[(int64_t)k * N + t] : det_cov[(int64_t)k * B + (t - N)]; }
    __device__ float ft(int t, int k) const
    {
        return t < N ? ent_feat[(int64_t)t * F + k] : det_feat[(int64_t)(t - N) * F + k];
    }
    __device__ float w(int t) const { return t < N ? ent_w[t] : 1.f; }
};

// pass 1: w, w (mu - c_g), w f into the winner g (acc arrays zeroed)
__global__ void assoc_sum1_kernel(Slots sl, const int32_t *__restrict__ parent, float *acc_w, float *acc_m,
                                  float *acc_f)
{
    const int T = sl.N + sl.B;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)T * (4 + sl.F)) return;
    const int t = (int)(i / (4 + sl.F)), k = (int)(i - (int64_t)t * (4 + sl.F));
    const int g = parent[t];
    const float w = sl.w(t);
    if (k == 0) atomicAdd(&acc_w[g], w);
    else if (k < 4) atomicAdd(&acc_m[(int64_t)(k - 1) * T + g], w * (sl.mu(t, k - 1) - sl.mu(g, k - 1)));
    else atomicAdd(&acc_f[(int64_t)g * sl.F + (k - 4)], w * sl.ft(t, k - 4));
}

// finalise the means and features of the winners
__global__ void assoc_fin1_kernel(Slots sl, const int32_t *__restrict__ parent, const float *__restrict__ acc_w,
                                  const float *__restrict__ acc_m, const float *__restrict__ acc_f, float *out_w,
                                  float *out_mu, float *out_feat)
{
    const int T = sl.N + sl.B;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)T * (4 + sl.F)) return;
    const int t = (int)(i / (4 + sl.F)), k = (int)(i - (int64_t)t * (4 + sl.F));
    const bool own = parent[t] == t && acc_w[t] > 0.f;
    if (k == 0) out_w[t] = own ? acc_w[t] : 0.f;
    else if (k < 4) out_mu[(int64_t)(k - 1) * T + t] = own ? sl.mu(t, k - 1) + acc_m[(int64_t)(k - 1) * T + t] / acc_w[t] : 0.f;
    else out_feat[(int64_t)t * sl.F + (k - 4)] = own ? acc_f[(int64_t)t * sl.F + (k - 4)] / acc_w[t] : 0.f;
}

// pass 2: w (S + (mu - mu_g)(mu - mu_g)') into the winner
__global__ void assoc_sum2_kernel(Slots sl, const int32_t *__restrict__ parent, const float *__restrict__ out_mu,
                                  float *acc_c)
{
    const int T = sl.N + sl.B;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= T) return;
    const int g = parent[t];
    const float w = sl.w(t);
    float dm[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) dm[k] = sl.mu(t, k) - out_mu[(int64_t)k * T + g];
    const int ia[6] = {0, 0, 0, 1, 1, 2}, ib[6] = {0, 1, 2, 1, 2, 2};
#pragma unroll
    for (int k = 0; k < 6; ++k) atomicAdd(&acc_c[(int64_t)k * T + g], w * (sl.cv(t, k) + dm[ia[k]] * dm[ib[k]]));
}

__global__ void assoc_fin2_kernel(int32_t T, const int32_t *__restrict__ parent, const float *__restrict__ acc_w,
                                  const float *__restrict__ acc_c, float *out_cov)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)T * 6) return;
    const int t = (int)(i / 6), k = (int)(i - (int64_t)t * 6);
    const bool own = parent[t] == t && acc_w[t] > 0.f;
    out_cov[(int64_t)k * T + t] = own ? acc_c[(int64_t)k * T + t] / acc_w[t] : 0.f;
}

}  // namespace

cudaError_t launch_assoc(const AssocArgs &a, cudaStream_t s)
{
    const int32_t N = a.N, B = a.B, F = a.F, T = a.N + a.B;
    if (B < 1 || N < 0 || F < 1 || a.max_m < 1 || (int64_t)B * a.max_m > 0x7fffffff) return cudaErrorInvalidValue;
    cudaError_t e;
    assoc_search_kernel<<<B, TA, 0, s>>>(a.S, a.ld, N, B, a.ent_mu, a.ent_cov, a.ent_active, a.det_mu, a.det_cov,
                                         a.tau_f, a.h_max, a.max_m, a.match_cnt, a.match_idx, a.match_h, a.err);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    // the labels in shared memory when they fit (up to 200 KB: 51,200 nodes)
    const size_t lab_bytes = (size_t)T * sizeof(int32_t);
    const int32_t in_smem = lab_bytes <= 200 * 1024 ? 1 : 0;
    if (in_smem && lab_bytes > 48 * 1024 &&
        (e = cudaFuncSetAttribute(assoc_components_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  200 * 1024)) != cudaSuccess)
        return e;
    assoc_components_kernel<<<1, 1024, in_smem ? lab_bytes : 0, s>>>(N, B, a.max_m, a.match_idx, a.label, 256,
                                                                     a.err, in_smem);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(a.win, 0, (size_t)T * sizeof(unsigned long long), s)) != cudaSuccess) return e;
    if (N > 0) {
        assoc_winner_kernel<<<(N + 255) / 256, 256, 0, s>>>(N, a.ent_w, a.label, a.win);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    assoc_parent_kernel<<<(T + 255) / 256, 256, 0, s>>>(T, a.label, a.win, a.parent);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(a.acc, 0, (size_t)T * (10 + F) * sizeof(float), s)) != cudaSuccess) return e;
    float *acc_w = a.acc, *acc_m = a.acc + T, *acc_c = a.acc + 4 * (int64_t)T, *acc_f = a.acc + 10 * (int64_t)T;
    const Slots sl{N, B, F, a.ent_mu, a.ent_cov, a.ent_feat, a.ent_w, a.det_mu, a.det_cov, a.det_feat};
    const int64_t n1 = (int64_t)T * (4 + F);
    assoc_sum1_kernel<<<(unsigned)((n1 + 255) / 256), 256, 0, s>>>(sl, a.parent, acc_w, acc_m, acc_f);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    assoc_fin1_kernel<<<(unsigned)((n1 + 255) / 256), 256, 0, s>>>(sl, a.parent, acc_w, acc_m, acc_f, a.out_w,
                                                                   a.out_mu, a.out_feat);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    assoc_sum2_kernel<<<(T + 255) / 256, 256, 0, s>>>(sl, a.parent, a.out_mu, acc_c);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    assoc_fin2_kernel<<<(unsigned)(((int64_t)T * 6 + 255) / 256), 256, 0, s>>>(T, a.parent, acc_w, acc_c, a.out_cov);
    return cudaGetLastError();
}

}  // namespace farm
