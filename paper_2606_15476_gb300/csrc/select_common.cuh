// select_common.cuh -- building blocks of the per-row rank selection
// (App. D.2 step 3 ranks, step 4 landmark candidates), shared by the
// shared-memory / chunked select (k_select.cu) and the thresholded select
// (k_select_thresh.cu).
//
// A row's entries map to order-preserving 32-bit keys; a candidate is the
// 64-bit word (key << 32) | (2^32 - 1 - position), so sorting words in
// descending order gives value descending, lower position first: the rank
// order of the definition
//   rank(j) = 1 + #{j' : c_j' > c_j, or c_j' = c_j and j' < j}.
// TH is the block size of the calling kernel.
#pragma once

#include "farm_internal.h"

namespace farm {
namespace sel {

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

__device__ __forceinline__ uint64_t cand_word(uint32_t key, int32_t pos)
{
    return ((uint64_t)key << 32) | (uint64_t)(0xffffffffu - (uint32_t)pos);
}

// Rank-ordered candidate words -> indices / values [0, stride); the object
// index of position p is idx_map[p] when idx_map is given, else
// idx_base + p.  Entries past R hold index -1 and value pad.
template <int TH>
__device__ __forceinline__ void write_list(const uint64_t *cand, int R, int32_t idx_base,
                                           const int32_t *__restrict__ idx_map, int32_t *__restrict__ oi,
                                           float *__restrict__ oc, int stride, float pad)
{
    for (int i = threadIdx.x; i < stride; i += TH) {
        if (i < R) {
            const uint64_t c = cand[i];
            const int32_t pos = (int32_t)(0xffffffffu - (uint32_t)(c & 0xffffffffu));
            oi[i] = idx_map ? idx_map[pos] : idx_base + pos;
            if (oc) oc[i] = key_value((uint32_t)(c >> 32));
        } else {
            oi[i] = -1;
            if (oc) oc[i] = pad;
        }
    }
}

// Descending bucket search over NB bins (NB a multiple of TH): the bin
// holding the `remaining`-th largest entry, how many of its entries are still
// needed, and its count.  Ends with a barrier; results in *s_bin, *s_rem,
// *s_cnt.
template <int NB, int TH>
__device__ __forceinline__ void find_bucket(const uint32_t *hist, uint32_t remaining, uint32_t *wsum,
                                            uint32_t *s_bin, uint32_t *s_rem, uint32_t *s_cnt)
{
    constexpr int BPT = NB / TH;    // bins per thread, highest bins to thread 0
    static_assert(BPT >= 1 && BPT * TH == NB, "bins per thread");
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

// The key of the R-th largest of n keys in shared memory (1 <= R <= n):
// three radix passes of 11, 11 and 10 bits.  hist: 2048 words of shared
// memory, wsum: TH / 32 words, s3: three words.
template <int TH>
__device__ __forceinline__ uint32_t kth_key(const uint32_t *keys, int n, int R, uint32_t *hist, uint32_t *wsum,
                                            uint32_t *s3)
{
    const int tid = threadIdx.x;
    uint32_t prefix = 0;
    uint32_t remaining = (uint32_t)R;
#pragma unroll 1
    for (int pass = 0; pass < 3; ++pass) {
        const int shift = pass == 0 ? 21 : (pass == 1 ? 10 : 0);
        const int nb = pass == 2 ? 1024 : 2048;
        const uint32_t pmask = pass == 0 ? 0u : (pass == 1 ? 0xffe00000u : 0xfffffc00u);
        for (int i = tid; i < nb; i += TH) hist[i] = 0;
        __syncthreads();
        for (int j = tid; j < n; j += TH) {
            const uint32_t k = keys[j];
            if ((k & pmask) == prefix) atomicAdd(&hist[(k >> shift) & (uint32_t)(nb - 1)], 1u);
        }
        __syncthreads();
        if (pass == 2) find_bucket<1024, TH>(hist, remaining, wsum, &s3[0], &s3[1], &s3[2]);
        else find_bucket<2048, TH>(hist, remaining, wsum, &s3[0], &s3[1], &s3[2]);
        prefix |= s3[0] << shift;
        remaining = s3[1];
        __syncthreads();   // s3 is rewritten by the next pass
    }
    return prefix;
}

// Bitonic sort of P (a power of two) candidate words in shared memory,
// descending.
template <int TH>
__device__ __forceinline__ void bitonic_desc(uint64_t *cand, int P)
{
    const int tid = threadIdx.x;
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
}

// Exact select of the R largest entries of one row read from global memory
// (four 8-bit radix passes over the row, then the ordered tie pass), written
// in rank order by write_list.  cand: at least the next power of two >= R
// words of shared memory; hist: 256 words; s_misc: TH / 32 + 3 words.
template <int TH>
__device__ __forceinline__ void select_row_global(const float *__restrict__ row, int n, int R, uint64_t *cand,
                                                  uint32_t *hist, int *s_misc, int32_t *__restrict__ oi,
                                                  float *__restrict__ oc, int out_stride, float pad)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    int *s_warp = s_misc;                       // TH / 32
    int *s_remaining = s_misc + TH / 32;
    int *s_cnt = s_remaining + 1;
    uint32_t *s_prefix = reinterpret_cast<uint32_t *>(s_cnt + 1);
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
            const uint32_t before = incl - sum;
            if (before < (uint32_t)remaining && incl >= (uint32_t)remaining) {
                uint32_t cum = before;
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    if (cum + loc[i] >= (uint32_t)remaining) {
                        *s_prefix = prefix | ((255u - (uint32_t)(lane * 8 + i)) << shift);
                        *s_remaining = remaining - (int)cum;
                        break;
                    }
                    cum += loc[i];
                }
            }
        }
        __syncthreads();
        prefix = *s_prefix;
        remaining = *s_remaining;
        mask |= 255u << shift;
        __syncthreads();
    }
    const uint32_t T = prefix;
    const int n_gt = R - remaining;   // entries strictly above T, all kept
    if (tid == 0) *s_cnt = 0;
    __syncthreads();
    for (int j = tid; j < n; j += TH) {
        const uint32_t k = order_key(row[j]);
        if (k > T) cand[atomicAdd(s_cnt, 1)] = cand_word(k, j);
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
            if (pos < remaining) cand[n_gt + pos] = cand_word(T, j);
        }
        taken += tot;
        __syncthreads();
    }
    int P = 1;
    while (P < R) P <<= 1;
    for (int i = R + tid; i < P; i += TH) cand[i] = 0ull;
    __syncthreads();
    bitonic_desc<TH>(cand, P);
    write_list<TH>(cand, R, 0, nullptr, oi, oc, out_stride, pad);
    __syncthreads();
}

}  // namespace sel
}  // namespace farm
