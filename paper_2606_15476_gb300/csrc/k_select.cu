// k_select.cu -- per-row rank selection (App. D.2 step 3 ranks, step 4
// landmark candidates).
//
// For each similarity row the kernel returns the R largest entries in rank
// order: value descending, lower object index first among equal values, i.e.
// exactly the objects of rank 1..R of the definition
//   rank(j) = 1 + #{j' : c_j' > c_j, or c_j' = c_j and j' < j}.
// Target rows keep R = r_tgt candidates (the rank bound of farm_query_batch),
// landmark rows keep R = K_a.
//
// One CTA per row.  Values map to order-preserving 32-bit keys; radix passes
// find the key T of the R-th largest entry and how many entries equal to T
// still belong in the list; one pass appends every key > T (and the entries
// equal to T when all of them belong); otherwise an ordered pass takes the
// first entries equal to T in index order; a bitonic sort over (key, index)
// in shared memory puts the list in rank order.
//
// Rows of up to kRowSmemMax entries are staged once in shared memory (two
// CTAs per SM) and take three passes with 11/11/10-bit digits over shared
// memory; longer rows stay in global memory (four 8-bit passes, L2-resident).
#include "farm_internal.h"

namespace farm {
namespace {

constexpr int TH = 512;
constexpr int SORT_MAX = kMaxTargetCands;   // >= kMaxAnchorCands
constexpr int kRowSmemMax = 24576;          // entries staged in shared memory (96 KB)

__device__ __forceinline__ uint32_t order_key(float f)
{
    const uint32_t u = __float_as_uint(f + 0.0f);   // -0 -> +0
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

__device__ __forceinline__ float key_value(uint32_t k)
{
    const uint32_t u = (k & 0x80000000u) ? (k & 0x7fffffffu) : ~k;
    return __uint_as_float(u);
}

__global__ void __launch_bounds__(TH)
select_rows_global_kernel(const float *__restrict__ S, int64_t ld_s, int32_t n, int64_t n_tgt_rows,
                   int32_t r_tgt, int32_t k_lm, int32_t *__restrict__ tsel_idx,
                   float *__restrict__ tsel_cos, int64_t tsel_row0, int32_t stride_t,
                   int32_t *__restrict__ lsel_idx, float *__restrict__ lsel_cos, int64_t lsel_row0,
                   int32_t stride_l)
{
    __shared__ uint32_t hist[256];
    __shared__ uint64_t cand[SORT_MAX];
    __shared__ uint32_t s_prefix;
    __shared__ int s_remaining, s_cnt, s_warp[TH / 32];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t r = blockIdx.x;
    const float *row = S + r * ld_s;
    const bool is_tgt = r < n_tgt_rows;
    const int R = is_tgt ? r_tgt : k_lm;

    uint32_t prefix = 0, mask = 0;
    int remaining = R;
    for (int shift = 24; shift >= 0; shift -= 8) {
        for (int i = tid; i < 256; i += TH) hist[i] = 0;
        __syncthreads();
        for (int j = tid; j < n; j += TH) {
            const uint32_t k = order_key(row[j]);
            if ((k & mask) == prefix) atomicAdd(&hist[(k >> shift) & 255u], 1u);
        }
        __syncthreads();
        if (warp == 0) {
            // suffix sums over 256 buckets: lane l owns buckets 255-8l .. 248-8l
            uint32_t loc[8], sum = 0;
#pragma unroll
            for (int i = 0; i < 8; ++i) { loc[i] = hist[255 - (lane * 8 + i)]; sum += loc[i]; }
            uint32_t incl = sum;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += v;
            }
            uint32_t before = incl - sum;   // entries in higher buckets than this lane's
            // the lane whose range crosses `remaining` finds the bucket
            if (before < (uint32_t)remaining && incl >= (uint32_t)remaining) {
                uint32_t cum = before;
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    if (cum + loc[i] >= (uint32_t)remaining) {
                        const uint32_t b = 255u - (uint32_t)(lane * 8 + i);
                        s_prefix = prefix | (b << shift);
                        s_remaining = remaining - (int)cum;
                        break;
                    }
                    cum += loc[i];
                }
            }
        }
        __syncthreads();
        prefix = s_prefix;
        remaining = s_remaining;
        mask |= 255u << shift;
    }
    const uint32_t T = prefix;
    const int n_gt = R - remaining;   // entries strictly above T, all kept

    if (tid == 0) s_cnt = 0;
    __syncthreads();
    for (int j = tid; j < n; j += TH) {
        const uint32_t k = order_key(row[j]);
        if (k > T) {
            const int pos = atomicAdd(&s_cnt, 1);
            cand[pos] = ((uint64_t)k << 32) | (uint64_t)(0xffffffffu - (uint32_t)j);
        }
    }
    __syncthreads();
    // the first `remaining` entries equal to T, in index order
    int taken = 0;
    for (int base = 0; base < n && taken < remaining; base += TH) {
        const int j = base + tid;
        const bool eq = j < n && order_key(row[j]) == T;
        const unsigned bal = __ballot_sync(0xffffffffu, eq);
        if (lane == 0) s_warp[warp] = __popc(bal);
        __syncthreads();
        int off = 0, tot = 0;
        for (int w = 0; w < TH / 32; ++w) {
            if (w < warp) off += s_warp[w];
            tot += s_warp[w];
        }
        if (eq) {
            const int pos = taken + off + __popc(bal & ((1u << lane) - 1u));
            if (pos < remaining)
                cand[n_gt + pos] = ((uint64_t)T << 32) | (uint64_t)(0xffffffffu - (uint32_t)j);
        }
        taken += tot;
        __syncthreads();
    }
    // bitonic sort, descending, over the next power of two >= R
    int P = 1;
    while (P < R) P <<= 1;
    for (int i = R + tid; i < P; i += TH) cand[i] = 0ull;
    __syncthreads();
    for (int k = 2; k <= P; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = tid; i < P; i += TH) {
                const int ixj = i ^ j;
                if (ixj > i) {
                    const uint64_t a = cand[i], b = cand[ixj];
                    const bool desc = (i & k) == 0;
                    if (desc ? (a < b) : (a > b)) { cand[i] = b; cand[ixj] = a; }
                }
            }
            __syncthreads();
        }
    }
    if (is_tgt) {
        int32_t *oi = tsel_idx + (tsel_row0 + r) * (int64_t)stride_t;
        float *oc = tsel_cos ? tsel_cos + (tsel_row0 + r) * (int64_t)stride_t : nullptr;
        for (int i = tid; i < stride_t; i += TH) {
            if (i < R) {
                const uint64_t c = cand[i];
                oi[i] = (int32_t)(0xffffffffu - (uint32_t)(c & 0xffffffffu));
                if (oc) oc[i] = key_value((uint32_t)(c >> 32));
            } else {
                oi[i] = -1;
                if (oc) oc[i] = 0.f;
            }
        }
    } else {
        int32_t *oi = lsel_idx + (lsel_row0 + (r - n_tgt_rows)) * (int64_t)stride_l;
        float *oc = lsel_cos ? lsel_cos + (lsel_row0 + (r - n_tgt_rows)) * (int64_t)stride_l : nullptr;
        for (int i = tid; i < stride_l; i += TH) {
            oi[i] = i < R ? (int32_t)(0xffffffffu - (uint32_t)(cand[i] & 0xffffffffu)) : -1;
            if (oc) oc[i] = i < R ? key_value((uint32_t)(cand[i] >> 32)) : 0.f;
        }
    }
}


// Descending bucket search over NB bins: the bin holding the `remaining`-th
// largest entry, how many of its entries are still needed, and its count.
template <int NB>
__device__ __forceinline__ void find_bucket(const uint32_t *hist, uint32_t remaining, uint32_t *wsum,
                                            uint32_t *s_bin, uint32_t *s_rem, uint32_t *s_cnt)
{
    constexpr int BPT = NB / TH;    // bins per thread, highest bins to thread 0
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    uint32_t loc[BPT], sum = 0;
#pragma unroll
    for (int i = 0; i < BPT; ++i) { loc[i] = hist[NB - 1 - (tid * BPT + i)]; sum += loc[i]; }
    uint32_t incl = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    uint32_t wbase = 0;
    for (int w = 0; w < warp; ++w) wbase += wsum[w];
    const uint32_t before = wbase + incl - sum;
    if (before < remaining && before + sum >= remaining) {
        uint32_t cum = before;
#pragma unroll
        for (int i = 0; i < BPT; ++i) {
            if (cum + loc[i] >= remaining) {
                *s_bin = (uint32_t)(NB - 1 - (tid * BPT + i));
                *s_rem = remaining - cum;
                *s_cnt = loc[i];
                break;
            }
            cum += loc[i];
        }
    }
    __syncthreads();
}

// Bitonic sort of P (a power of two <= TH) 64-bit keys in shared memory,
// descending, one element per thread.  Stages whose partners lie in the same
// warp synchronise the warp only.
__device__ __forceinline__ void bitonic_desc(uint64_t *cand, int P)
{
    const int i = threadIdx.x;
    int prev_j = TH;
    for (int k = 2; k <= P; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            if (j >= 32 || prev_j >= 32) __syncthreads();
            else __syncwarp();
            if (i < P) {
                const int ixj = i ^ j;
                if (ixj > i) {
                    const uint64_t a = cand[i], b = cand[ixj];
                    const bool desc = (i & k) == 0;
                    if (desc ? (a < b) : (a > b)) { cand[i] = b; cand[ixj] = a; }
                }
            }
            prev_j = j;
        }
    }
    __syncthreads();
}

constexpr int kVecHalf = kRowSmemMax / 8 / TH;   // float4 loads per thread per batch (two batches)

__global__ void __launch_bounds__(TH, 2)
select_rows_smem_kernel(const float *__restrict__ S, int64_t ld_s, int32_t n, int64_t n_tgt_rows,
                        int32_t r_tgt, int32_t k_lm, int32_t *__restrict__ tsel_idx,
                        float *__restrict__ tsel_cos, int64_t tsel_row0, int32_t stride_t,
                        int32_t *__restrict__ lsel_idx, float *__restrict__ lsel_cos, int64_t lsel_row0,
                   int32_t stride_l)
{
    extern __shared__ uint32_t keys[];
    __shared__ uint32_t hist[2048];
    __shared__ uint64_t cand[SORT_MAX];
    __shared__ uint32_t wsum[TH / 32];
    __shared__ uint32_t s_bin, s_rem, s_cnt;
    __shared__ int s_app, s_warp[TH / 32];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t r = blockIdx.x;
    const float *row = S + r * ld_s;
    const bool is_tgt = r < n_tgt_rows;
    const int R = is_tgt ? r_tgt : k_lm;
    const int n4 = n & ~3;

    // issue the row's loads in two batches of kVecHalf float4 per thread, then
    // histogram the top 11 bits of each key
    for (int i = tid; i < 2048; i += TH) hist[i] = 0;
    __syncthreads();
#pragma unroll
    for (int half = 0; half < 2; ++half) {
        float4 buf[kVecHalf];
#pragma unroll
        for (int u = 0; u < kVecHalf; ++u) {
            const int i = ((half * kVecHalf + u) * TH + tid) * 4;
            buf[u] = i < n4 ? __ldg(reinterpret_cast<const float4 *>(row + i)) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int u = 0; u < kVecHalf; ++u) {
            const int i = ((half * kVecHalf + u) * TH + tid) * 4;
            if (i < n4) {
                const uint4 k = make_uint4(order_key(buf[u].x), order_key(buf[u].y), order_key(buf[u].z),
                                           order_key(buf[u].w));
                *reinterpret_cast<uint4 *>(keys + i) = k;
                atomicAdd(&hist[k.x >> 21], 1u);
                atomicAdd(&hist[k.y >> 21], 1u);
                atomicAdd(&hist[k.z >> 21], 1u);
                atomicAdd(&hist[k.w >> 21], 1u);
            }
        }
    }
    if (tid < n - n4) {
        const uint32_t k = order_key(row[n4 + tid]);
        keys[n4 + tid] = k;
        atomicAdd(&hist[k >> 21], 1u);
    }
    __syncthreads();
    find_bucket<2048>(hist, (uint32_t)R, wsum, &s_bin, &s_rem, &s_cnt);
    const uint32_t b1 = s_bin;
    uint32_t remaining = s_rem;
    const int nv = (n + 3) >> 2;   // uint4 groups (the tail group is masked by index)
    // second digit: bits 10..20 among keys whose top digit is b1
    for (int i = tid; i < 2048; i += TH) hist[i] = 0;
    __syncthreads();
    for (int g = tid; g < nv; g += TH) {
        const uint4 k = reinterpret_cast<const uint4 *>(keys)[g];
        const uint32_t kk[4] = {k.x, k.y, k.z, k.w};
#pragma unroll
        for (int c = 0; c < 4; ++c)
            if (4 * g + c < n && (kk[c] >> 21) == b1) atomicAdd(&hist[(kk[c] >> 10) & 2047u], 1u);
    }
    __syncthreads();
    find_bucket<2048>(hist, remaining, wsum, &s_bin, &s_rem, &s_cnt);
    const uint32_t p2 = (b1 << 11) | s_bin;     // top 22 bits
    remaining = s_rem;
    // third digit: bits 0..9
    for (int i = tid; i < 1024; i += TH) hist[i] = 0;
    __syncthreads();
    for (int g = tid; g < nv; g += TH) {
        const uint4 k = reinterpret_cast<const uint4 *>(keys)[g];
        const uint32_t kk[4] = {k.x, k.y, k.z, k.w};
#pragma unroll
        for (int c = 0; c < 4; ++c)
            if (4 * g + c < n && (kk[c] >> 10) == p2) atomicAdd(&hist[kk[c] & 1023u], 1u);
    }
    __syncthreads();
    find_bucket<1024>(hist, remaining, wsum, &s_bin, &s_rem, &s_cnt);
    const uint32_t T = (p2 << 10) | s_bin;
    remaining = s_rem;
    const bool take_all_eq = s_cnt == remaining;
    const int n_gt = R - (int)remaining;

    if (tid == 0) s_app = 0;
    __syncthreads();
    for (int g = tid; g < nv; g += TH) {
        const uint4 k = reinterpret_cast<const uint4 *>(keys)[g];
        const uint32_t kk[4] = {k.x, k.y, k.z, k.w};
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int i = 4 * g + c;
            if (i < n && (kk[c] > T || (take_all_eq && kk[c] == T))) {
                const int pos = atomicAdd(&s_app, 1);
                cand[pos] = ((uint64_t)kk[c] << 32) | (uint64_t)(0xffffffffu - (uint32_t)i);
            }
        }
    }
    __syncthreads();
    if (!take_all_eq) {
        int taken = 0;
        for (int base = 0; base < n && taken < (int)remaining; base += TH) {
            const int j = base + tid;
            const bool eq = j < n && keys[j] == T;
            const unsigned bal = __ballot_sync(0xffffffffu, eq);
            if (lane == 0) s_warp[warp] = __popc(bal);
            __syncthreads();
            int off = 0, tot = 0;
            for (int w = 0; w < TH / 32; ++w) {
                if (w < warp) off += s_warp[w];
                tot += s_warp[w];
            }
            if (eq) {
                const int pos = taken + off + __popc(bal & ((1u << lane) - 1u));
                if (pos < (int)remaining)
                    cand[n_gt + pos] = ((uint64_t)T << 32) | (uint64_t)(0xffffffffu - (uint32_t)j);
            }
            taken += tot;
            __syncthreads();
        }
    }
    int P = 1;
    while (P < R) P <<= 1;
    for (int i = R + tid; i < P; i += TH) cand[i] = 0ull;
    bitonic_desc(cand, P);
    if (is_tgt) {
        int32_t *oi = tsel_idx + (tsel_row0 + r) * (int64_t)stride_t;
        float *oc = tsel_cos ? tsel_cos + (tsel_row0 + r) * (int64_t)stride_t : nullptr;
        for (int i = tid; i < stride_t; i += TH) {
            if (i < R) {
                const uint64_t c = cand[i];
                oi[i] = (int32_t)(0xffffffffu - (uint32_t)(c & 0xffffffffu));
                if (oc) oc[i] = key_value((uint32_t)(c >> 32));
            } else {
                oi[i] = -1;
                if (oc) oc[i] = 0.f;
            }
        }
    } else {
        int32_t *oi = lsel_idx + (lsel_row0 + (r - n_tgt_rows)) * (int64_t)stride_l;
        float *oc = lsel_cos ? lsel_cos + (lsel_row0 + (r - n_tgt_rows)) * (int64_t)stride_l : nullptr;
        for (int i = tid; i < stride_l; i += TH) {
            oi[i] = i < R ? (int32_t)(0xffffffffu - (uint32_t)(cand[i] & 0xffffffffu)) : -1;
            if (oc) oc[i] = i < R ? key_value((uint32_t)(cand[i] >> 32)) : 0.f;
        }
    }
}

}  // namespace

cudaError_t launch_select_rows_ex(const float *S, int64_t ld_s, int64_t n, int64_t rows, int64_t n_tgt_rows,
                                  int32_t r_tgt, int32_t k_lm, int32_t *tsel_idx, float *tsel_cos, int64_t tsel_row0,
                                  int32_t stride_t, int32_t *lsel_idx, float *lsel_cos, int64_t lsel_row0,
                                  int32_t stride_l, cudaStream_t s)
{
    if (rows <= 0) return cudaSuccess;
    if (r_tgt < 1 || r_tgt > SORT_MAX || r_tgt > n || k_lm < 1 || k_lm > kMaxAnchorCands ||
        k_lm > n || n > 0x7fffffff)
        return cudaErrorInvalidValue;
    if (n <= kRowSmemMax && (ld_s % 4) == 0 && ((uintptr_t)S & 15u) == 0) {
        const size_t smem = (size_t)((n + 3) & ~3) * sizeof(uint32_t);
        cudaError_t e = cudaFuncSetAttribute(select_rows_smem_kernel,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        select_rows_smem_kernel<<<(unsigned)rows, TH, smem, s>>>(S, ld_s, (int32_t)n, n_tgt_rows, r_tgt, k_lm,
                                                                  tsel_idx, tsel_cos, tsel_row0, stride_t,
                                                                  lsel_idx, lsel_cos, lsel_row0, stride_l);
    } else {
        select_rows_global_kernel<<<(unsigned)rows, TH, 0, s>>>(S, ld_s, (int32_t)n, n_tgt_rows, r_tgt, k_lm,
                                                                 tsel_idx, tsel_cos, tsel_row0, stride_t,
                                                                 lsel_idx, lsel_cos, lsel_row0, stride_l);
    }
    return cudaGetLastError();
}

cudaError_t launch_select_rows(const float *S, int64_t ld_s, int64_t n, int64_t rows,
                               int64_t n_tgt_rows, int32_t r_tgt, int32_t k_lm,
                               int32_t *tsel_idx, float *tsel_cos, int64_t tsel_row0,
                               int32_t stride_t, int32_t *lsel_idx, int64_t lsel_row0,
                               int32_t stride_l, cudaStream_t s)
{
    return launch_select_rows_ex(S, ld_s, n, rows, n_tgt_rows, r_tgt, k_lm, tsel_idx, tsel_cos, tsel_row0, stride_t,
                                 lsel_idx, nullptr, lsel_row0, stride_l, s);
}

}  // namespace farm
