// k_fuse_select.cu -- the rank selection fused with the similarity kernel
// (App. D.2 step 3 ranks, step 4 landmark candidates), so that the
// similarity block S is never written.
//
// For each row the R largest entries are wanted (R = the row's list length),
// in the rank order of the definition: value descending, lower object index
// first.  Let every entry be the 64-bit word (order key << 32) | (2^32 - 1 -
// index); then the rank order is the word order, all words are distinct,
// and the R best entries are the R largest words.
//
// 1. A sample of the row -- the tiles 0, s, 2s, ... of 256 objects -- is
//    computed first (the similarity kernel in its sample mode: values stored
//    compacted, with the maximum of every group of 8 or 32 of them).
// 2. sample_tau (below) takes the R-th largest of the sample's group maxima
//    (of its values when the groups are fewer than R) as a bound tau0.  The
//    group maxima are entries of the row, and a subset cannot have a larger
//    R-th element: tau0 <= the row's R-th largest value.  It appends the
//    sample's own entries >= tau0 to the row's candidate buffer and sets the
//    row's threshold tau to the R-th largest of those (= the sample's R-th
//    largest value, again at most the row's), so every one of the row's R
//    best entries outside the sample is >= tau.
// 3. The similarity kernel runs over the other tiles and appends every entry
//    >= tau.  The buffer now holds every entry >= tau of the other tiles and
//    every sample entry >= tau0 (tau0 <= tau), hence the row's R best words.
// 4. fuse_final (below): the R largest words of the buffer, sorted, are the
//    row's rank list.  A row whose candidates overflowed the buffer is
//    recorded for the exact fallback.
//
// The threshold of step 2 may be optimistic: tau = the sample's k-th largest
// value for a k below R (optimistic_rank), which lets about k s of the row's
// entries through instead of R s (a sample of every s-th tile).  It is a lower bound of the row's R-th
// value exactly when at least R of the row's entries reach it, and then the
// buffer holds the R best words as above; fuse_final counts the buffer's
// words that reach tau and records a row with fewer than R for the exact
// fallback.  With the sample a random fraction f of the row, the count of
// entries reaching its k-th largest value is about negative-binomial, mean
// k / f; k is chosen so that the mean lies 4.5 deviations above R.
// 5. fuse_fallback (below) recomputes each recorded row over all its objects
//    (FP32 on the CUDA cores) and selects it exactly; with no recorded row it
//    returns at once.
//
// Two-pass rows (Piece::fs < 0; long rows of long lists, whose sample would
// have to be most of the row): step 1 computes every tile but stores only the
// group maxima; maxima_tau (below) takes the R-th largest of them as the
// threshold (a lower bound of the row's R-th value, as above) and the
// similarity kernel's second launch appends every entry of every tile that
// reaches it; steps 4-5 as above.  About R of the row's group maxima reach the
// threshold, so the appended entries number R and a few more per such group.
//
// One warp per row in sample_tau, maxima_tau and fuse_final, no block barriers.
#include <cuda_fp16.h>

#include "select_common.cuh"

namespace farm {
namespace {


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

// The piece holding launch row b, found by lane 0 and broadcast.
__device__ __forceinline__ int warp_find_piece(const Piece *__restrict__ pieces, int n_pieces, int64_t b)
{
    int lo = 0;
    if ((threadIdx.x & 31) == 0) {
        int hi = n_pieces - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (pieces[mid].row_begin <= b) lo = mid;
            else hi = mid - 1;
        }
    }
    return __shfl_sync(0xffffffffu, lo, 0);
}

struct RowList {
    int32_t *oi;
    float *oc;
    int stride, keep;
    int64_t grow;      // operand row (threshold, count, buffer)
};

// Launch row b's list (its whole-row length fkeep) and operand row.
__device__ __forceinline__ RowList row_list(const Piece &pc, int64_t b, int32_t *tsel_idx, float *tsel_cos,
                                            int32_t stride_t, int32_t *lsel_idx, float *lsel_cos, int32_t stride_l)
{
    const int i = (int)(b - pc.row_begin);
    RowList L;
    L.grow = pc.q_row0 + i;
    if (i < pc.ntr) {
        const int64_t o = (pc.t_row0 + i) * (int64_t)stride_t;
        L.oi = tsel_idx + o;
        L.oc = tsel_cos + o;
        L.stride = stride_t;
        L.keep = pc.fkeep_t;
    } else {
        const int64_t o = (pc.l_row0 + (i - pc.ntr)) * (int64_t)stride_l;
        L.oi = lsel_idx + o;
        L.oc = lsel_cos + o;
        L.stride = stride_l;
        L.keep = pc.fkeep_l;
    }
    return L;
}

// Keys staged per warp by sample_tau: the sample's group maxima, or its values
// when the groups are fewer than the list length -- at most this many, a
// prefix being still a subset of the row (small, so that many warps stay
// resident to hide the loads' latency).
constexpr int TAU_KEYS = 1024;
constexpr int TAU_WARPS = 4;
// Bits resolved by sample_tau's searches below the leading bits that the
// smallest and largest key share.  A threshold only has to be a lower bound
// of the row's R-th largest value, and a search stopped early returns one;
// 14 bits leave it within about 2^-12 (relative) of the exact R-th key,
// where a row holds few entries.
constexpr int TAU_BITS = 14;

// A lower bound of the R-th largest of n keys in shared memory (n >= R >= 1):
// the largest key T with at least R keys >= T among those whose bits below
// the shared leading bits are resolved to the first `bits` -- the exact R-th
// key when bits covers them all.  Stops as soon as exactly R keys reach the
// candidate (no further bit changes which keys do).  Never returns a key
// below that of -FLT_MAX other than 0 (every entry passes), so that its float
// value is a number.
__device__ __forceinline__ uint32_t warp_kth_lower(const uint32_t *keys, int n, int R, int bits, int lane)
{
    uint32_t kmin = 0xffffffffu, kmax = 0u;
    for (int j = lane; j < n; j += 32) {
        kmin = min(kmin, keys[j]);
        kmax = max(kmax, keys[j]);
    }
    kmin = __reduce_min_sync(0xffffffffu, kmin);
    kmax = __reduce_max_sync(0xffffffffu, kmax);
    const uint32_t diff = kmin ^ kmax;
    const int top = diff ? 31 - __clz(diff) : -1;
    uint32_t T = top < 0 ? kmin : (top == 31 ? 0u : kmin & ~((2u << top) - 1u));
    const int stop = top - bits;
    for (int bit = top; bit >= 0 && bit > stop; --bit) {
        const uint32_t c = T | (1u << bit);
        int cnt = 0;
        for (int j = lane; j < n; j += 32) cnt += keys[j] >= c ? 1 : 0;
        cnt = __reduce_add_sync(0xffffffffu, cnt);
        if (cnt >= R) {
            T = c;
            if (cnt == R) break;
        }
    }
    return T < 0x00800000u ? 0u : T;
}

// The sample rank whose value sets a row's optimistic threshold, for a list
// of R and a sample holding the fraction f of the row: the count of the row's
// entries reaching the sample's k-th largest is about negative-binomial, mean
// k / f and deviation sqrt(k (1 - f)) / f, and k is the smallest whose mean
// lies 4.5 deviations above R -- k = x^2 with x^2 - 4.5 sqrt(1 - f) x = R f --
// at most R (a sample that is the whole row: k = R, exact).
__device__ __forceinline__ int optimistic_rank(int R, int sample_n, int row_n)
{
    const float f = fminf(1.f, (float)sample_n / (float)row_n);
    const float a = 4.5f * sqrtf(1.f - f);
    const float x = 0.5f * (a + sqrtf(a * a + 4.f * (float)R * f));
    const int k = (int)ceilf(x * x);
    return k < R ? k : R;
}

// Eight consecutive sample values of a lane from j (16-byte aligned), zero past n.
__device__ __forceinline__ void load8(const float *__restrict__ row, int j, int n, float (&x)[8])
{
    if (j + 8 <= n) {
        const float4 a = __ldg(reinterpret_cast<const float4 *>(row + j));
        const float4 c = __ldg(reinterpret_cast<const float4 *>(row + j + 4));
        x[0] = a.x; x[1] = a.y; x[2] = a.z; x[3] = a.w; x[4] = c.x; x[5] = c.y; x[6] = c.z; x[7] = c.w;
    } else {
#pragma unroll
        for (int u = 0; u < 8; ++u) x[u] = j + u < n ? __ldg(row + j + u) : 0.f;
    }
}

__global__ void __launch_bounds__(TAU_WARPS * 32)
sample_tau_kernel(const float *__restrict__ S, const float *__restrict__ tops, const Piece *__restrict__ pieces,
                  int32_t n_pieces, int64_t total_rows, FuseEmit emit)
{
    __shared__ uint32_t keys[TAU_WARPS][TAU_KEYS];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t b = (int64_t)blockIdx.x * TAU_WARPS + warp;
    if (b >= total_rows) return;
    const Piece pc = pieces[warp_find_piece(pieces, n_pieces, b)];
    if (pc.fs <= 0) return;                    // a row of the unfused path, or a two-pass row
    const int s = pc.fs;
    const int i = (int)(b - pc.row_begin);
    const int64_t grow = pc.q_row0 + i;
    const int R = i < pc.ntr ? pc.fkeep_t : pc.fkeep_l;
    const int n = pc.n;                        // valid entries of the sample row
    const float *row = S + pc.s_off + (int64_t)i * pc.ld;
    uint32_t *kw = keys[warp];
    // the scan's first 16 values per lane are in flight during the search
    float xa[8], xb[8];
    load8(row, lane * 8, n, xa);
    load8(row, 256 + lane * 8, n, xb);
    const int G = (int)group_count(n, pc.gshift);
    uint32_t T = 0u;                           // key 0: every entry passes
    if (G >= R) {
        const float *tp = tops + pc.tops_off + (int64_t)i * group_stride(n, pc.gshift);
        const int g = min(G, TAU_KEYS);
#pragma unroll 4
        for (int j = lane; j < g; j += 32) kw[j] = order_key(__ldg(tp + j));
        __syncwarp();
        T = warp_kth_lower(kw, g, R, TAU_BITS, lane);
    } else if (n >= R) {
        const int g = min(n, TAU_KEYS);
#pragma unroll 4
        for (int j = lane; j < g; j += 32) kw[j] = order_key(__ldg(row + j));
        __syncwarp();
        T = g >= R ? warp_kth_lower(kw, g, R, TAU_BITS, lane) : 0u;
    }
    __syncwarp();
    // the sample's own entries >= tau (their positions mapped to objects),
    // their keys also staged: 8 consecutive entries per lane and chunk, the
    // next chunk's loads issued before this one's entries are placed; each
    // round places one entry of every lane that still holds one (a warp
    // ballot gives the places), so a chunk takes as many rounds as its
    // busiest lane has entries -- usually one or none
    const bool all = T == 0u;
    const float tf = key_value(T);             // entries >= tf are those whose key is >= T
    const uint32_t lt = (1u << lane) - 1u;
    uint64_t *dst = emit.cand + grow * (int64_t)emit.cap;
    int cnt = 0;
    for (int j0 = 0; j0 < n; j0 += 256) {
        const int jb = j0 + lane * 8;
        uint32_t take = 0u;
#pragma unroll
        for (int u = 0; u < 8; ++u) take |= (jb + u < n && (all || xa[u] >= tf)) ? (1u << u) : 0u;
        float cur[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) cur[u] = xa[u];
#pragma unroll
        for (int u = 0; u < 8; ++u) xa[u] = xb[u];
        if (j0 + 512 < n) load8(row, j0 + 512 + lane * 8, n, xb);
        while (__any_sync(0xffffffffu, take != 0u)) {
            const uint32_t bal = __ballot_sync(0xffffffffu, take != 0u);
            if (take) {
                const int u = __ffs(take) - 1;
                take &= take - 1u;
                float v = cur[0];
#pragma unroll
                for (int w = 1; w < 8; ++w) v = u == w ? cur[w] : v;
                const int pos = cnt + __popc(bal & lt);
                const int j = jb + u;
                const uint32_t k = order_key(v);
                const int32_t obj = (j >> 8) * s * 256 + (j & 255);
                if (pos < emit.cap) dst[pos] = ((uint64_t)k << 32) | (uint64_t)(0xffffffffu - (uint32_t)obj);
                if (pos < TAU_KEYS) kw[pos] = k;
            }
            cnt += __popc(bal);
        }
    }
    __syncwarp();
    // the threshold for the other tiles: the R-th largest of the sample's
    // entries themselves (at least tau, still at most the row's R-th value),
    // which keeps fewer of the other tiles' entries than the group bound
    // (optimistic: the sample's k-th largest entry, k <= R; fuse_final checks
    // that at least R of the row's entries reached it)
    const int k = optimistic_rank(R, n, pc.n_obj);
    if (T != 0u && cnt > k && cnt <= TAU_KEYS) T = max(T, warp_kth_lower(kw, cnt, k, TAU_BITS, lane));
    if (lane == 0) {
        emit.tau_key[grow] = T;
        emit.cnt[grow] = cnt;
    }
}

// A two-pass row's threshold: the R-th largest of its group maxima over the
// whole row (R its whole-row list length), staged in the warp's gmax keys of
// dynamic shared memory; every entry passes when the groups are fewer than R.
__global__ void __launch_bounds__(TAU_WARPS * 32)
maxima_tau_kernel(const float *__restrict__ tops, const Piece *__restrict__ pieces, int32_t n_pieces,
                  int64_t total_rows, FuseEmit emit, int32_t gmax)
{
    extern __shared__ uint32_t mkeys[];        // [TAU_WARPS][gmax]
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t b = (int64_t)blockIdx.x * TAU_WARPS + warp;
    if (b >= total_rows) return;
    const Piece pc = pieces[warp_find_piece(pieces, n_pieces, b)];
    if (pc.fs >= 0) return;                    // not a two-pass row
    const int i = (int)(b - pc.row_begin);
    const int64_t grow = pc.q_row0 + i;
    const int R = i < pc.ntr ? pc.fkeep_t : pc.fkeep_l;
    const int G = (int)group_count(pc.n, pc.gshift);
    uint32_t T = 0u;                           // key 0: every entry passes
    if (G >= R) {
        uint32_t *kw = mkeys + (int64_t)warp * gmax;
        const float *tp = tops + pc.tops_off + (int64_t)i * group_stride(pc.n, pc.gshift);
        const int g = min(G, gmax);            // (a prefix of the maxima still gives a lower bound)
#pragma unroll 4
        for (int j = lane; j < g; j += 32) kw[j] = order_key(__ldg(tp + j));
        __syncwarp();
        T = warp_kth_lower(kw, g, R, TAU_BITS, lane);
    }
    if (lane == 0) {
        emit.tau_key[grow] = T;
        emit.cnt[grow] = 0;
    }
}

// Whether at least `keep` of a row's t buffered words reach its threshold
// key T: the check of an optimistic threshold (a row that fails it is left
// to the exact fallback).
__device__ __forceinline__ bool threshold_held(const uint64_t *__restrict__ cand, int t, uint32_t T, int keep,
                                               int lane)
{
    int reach = 0;
    for (int j = lane; j < t; j += 32) reach += (uint32_t)(cand[j] >> 32) >= T ? 1 : 0;
    return (int)__reduce_add_sync(0xffffffffu, (unsigned)reach) >= keep;
}

// Merge of one row held in REG words per lane (REG * 32 >= total): the
// sample list's ms entries, then `total - ms` appended words from cand; the
// first keep of their word order written to the row's list.
template <int REG>
__device__ __forceinline__ void merge_row(const RowList &L, int ms, int total, const uint64_t *__restrict__ cand,
                                          uint64_t *cw, int lane)
{
    uint64_t w[REG];
#pragma unroll
    for (int k = 0; k < REG; ++k) {
        const int t = lane + 32 * k;
        uint64_t x = 0ull;    // no real word is 0 (its key would encode a NaN)
        if (t < ms) x = ((uint64_t)order_key(L.oc[t]) << 32) | (uint64_t)(0xffffffffu - (uint32_t)L.oi[t]);
        else if (t < total) x = cand[t - ms];
        w[k] = x;
    }
    __syncwarp();     // every lane has read the sample list before it is overwritten
    const int keep = total < L.keep ? total : L.keep;
    // T: the largest key with at least `keep` words at or above it, searched
    // below the leading bits that the smallest and largest keys share
    uint32_t T = 0u;
    if (total > keep) {
        uint32_t kmin = 0xffffffffu, kmax = 0u;
#pragma unroll
        for (int k = 0; k < REG; ++k) {
            if (w[k]) {
                const uint32_t key = (uint32_t)(w[k] >> 32);
                kmin = min(kmin, key);
                kmax = max(kmax, key);
            }
        }
        kmin = __reduce_min_sync(0xffffffffu, kmin);
        kmax = __reduce_max_sync(0xffffffffu, kmax);
        const uint32_t diff = kmin ^ kmax;
        const int top = diff ? 31 - __clz(diff) : -1;
        T = top < 0 ? kmin : (top == 31 ? 0u : kmin & ~((2u << top) - 1u));
#pragma unroll 1
        for (int bit = top; bit >= 0; --bit) {
            const uint32_t c = T | (1u << bit);
            int n = 0;
#pragma unroll
            for (int k = 0; k < REG; ++k) n += (uint32_t)(w[k] >> 32) >= c ? 1 : 0;
            n = __reduce_add_sync(0xffffffffu, n);
            if (n >= keep) {
                T = c;
                if (n == keep) break;     // no lower bit changes which words reach T
            }
        }
    }
    // collect the words at or above T (the keep best and their key ties)
    int nc = 0;
#pragma unroll
    for (int k = 0; k < REG; ++k) {
        const bool take = w[k] != 0ull && (uint32_t)(w[k] >> 32) >= T;
        const unsigned bal = __ballot_sync(0xffffffffu, take);
        if (take) cw[nc + __popc(bal & ((1u << lane) - 1u))] = w[k];
        nc += __popc(bal);
    }
    __syncwarp();
    // rank by counting (all words distinct); the first keep go to the list
    for (int j = lane; j < nc; j += 32) {
        const uint64_t x = cw[j];
        int rank = 0;
        for (int t = 0; t < nc; ++t) rank += cw[t] > x ? 1 : 0;
        if (rank < keep) {
            L.oi[rank] = (int32_t)(0xffffffffu - (uint32_t)(x & 0xffffffffu));
            L.oc[rank] = key_value((uint32_t)(x >> 32));
        }
    }
    for (int k = keep + lane; k < L.stride; k += 32) {
        L.oi[k] = -1;
        L.oc[k] = 0.f;
    }
}

// Rows of at most FINAL_SMALL words merge in fuse_final_kernel, FW warps
// (rows) per block, each row in the fewest registers its words need; a longer
// row (up to the buffer's capacity) is listed for fuse_final_big_kernel, whose
// warps hold up to 64 words a lane -- so that the common rows run at the
// occupancy of their own register count.
constexpr int FINAL_SMALL = 1024;
constexpr int FINAL_BIG_BLOCKS = 152;

template <int FW>
__global__ void __launch_bounds__(FW * 32)
fuse_final_kernel(const Piece *__restrict__ pieces, int32_t n_pieces, int64_t total_rows, int32_t *tsel_idx,
                  float *tsel_cos, int32_t stride_t, int32_t *lsel_idx, float *lsel_cos, int32_t stride_l,
                  FuseEmit emit, int32_t *n_overflow, int32_t *overflow_rows, int32_t *n_big, int32_t *big_rows)
{
    __shared__ uint64_t coll[FW][FINAL_SMALL];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t b = (int64_t)blockIdx.x * FW + warp;
    if (b >= total_rows) return;
    const Piece pc = pieces[warp_find_piece(pieces, n_pieces, b)];
    if (pc.fs == 0) return;                    // a row of the unfused path
    const RowList L = row_list(pc, b, tsel_idx, tsel_cos, stride_t, lsel_idx, lsel_cos, stride_l);
    const int32_t t = emit.cnt[L.grow];
    if (t > FINAL_SMALL) {
        // more candidates than the buffer holds: the exact fallback recomputes
        // the row; else the merge of long rows takes it
        if (lane == 0) {
            if (t > emit.cap) overflow_rows[atomicAdd(n_overflow, 1)] = (int32_t)b;
            else big_rows[atomicAdd(n_big, 1)] = (int32_t)b;
        }
        return;
    }
    const uint64_t *cand = emit.cand + L.grow * (int64_t)emit.cap;
    if (!threshold_held(cand, t, emit.tau_key[L.grow], L.keep, lane)) {
        if (lane == 0) overflow_rows[atomicAdd(n_overflow, 1)] = (int32_t)b;
        return;
    }
    if (t <= 128) merge_row<4>(L, 0, t, cand, coll[warp], lane);
    else if (t <= 256) merge_row<8>(L, 0, t, cand, coll[warp], lane);
    else if (t <= 512) merge_row<16>(L, 0, t, cand, coll[warp], lane);
    else merge_row<FINAL_SMALL / 32>(L, 0, t, cand, coll[warp], lane);
}

// The listed long rows (*n_big of them), a grid-stride loop of one-warp
// blocks; returns at once when none is listed.
template <int MAXR>
__global__ void __launch_bounds__(32)
fuse_final_big_kernel(const Piece *__restrict__ pieces, int32_t n_pieces, int32_t *tsel_idx, float *tsel_cos,
                      int32_t stride_t, int32_t *lsel_idx, float *lsel_cos, int32_t stride_l, FuseEmit emit,
                      const int32_t *__restrict__ n_big, const int32_t *__restrict__ big_rows, int32_t *n_overflow,
                      int32_t *overflow_rows)
{
    __shared__ uint64_t coll[MAXR * 32];
    const int lane = threadIdx.x;
    const int count = *n_big;
    for (int k = blockIdx.x; k < count; k += gridDim.x) {
        const int64_t b = big_rows[k];
        const Piece pc = pieces[warp_find_piece(pieces, n_pieces, b)];
        const RowList L = row_list(pc, b, tsel_idx, tsel_cos, stride_t, lsel_idx, lsel_cos, stride_l);
        const int32_t t = emit.cnt[L.grow];
        const uint64_t *cand = emit.cand + L.grow * (int64_t)emit.cap;
        if (threshold_held(cand, t, emit.tau_key[L.grow], L.keep, lane)) {
            merge_row<MAXR>(L, 0, t, cand, coll, lane);
        } else if (lane == 0) {
            overflow_rows[atomicAdd(n_overflow, 1)] = (int32_t)b;
        }
        __syncwarp();
    }
}

constexpr int FB_TH = 256;

__global__ void __launch_bounds__(FB_TH)
fuse_fallback_kernel(const Piece *__restrict__ pieces, int32_t n_pieces, const int32_t *__restrict__ n_overflow,
                     const int32_t *__restrict__ overflow_rows, const float *__restrict__ q32,
                     const uint16_t *__restrict__ q_hi, const uint16_t *__restrict__ q_lo, int32_t dim_pad,
                     int32_t *tsel_idx, float *tsel_cos, int32_t stride_t, int32_t *lsel_idx, float *lsel_cos,
                     int32_t stride_l, float *__restrict__ slab, int64_t slab_ld, int32_t *n_fallback)
{
    extern __shared__ float4 qs[];        // the row, dim_pad floats
    __shared__ uint64_t cand[kMaxTargetCands];
    __shared__ uint32_t hist[256];
    __shared__ int s_misc[FB_TH / 32 + 3];
    __shared__ int s_piece;
    const int tid = threadIdx.x;
    const int count = *n_overflow;
    if (blockIdx.x == 0 && tid == 0 && count > 0 && n_fallback) atomicAdd(n_fallback, count);
    float *row = slab + (int64_t)blockIdx.x * slab_ld;
    for (int k = blockIdx.x; k < count; k += gridDim.x) {
        const int64_t b = overflow_rows[k];
        if (tid == 0) {
            int lo = 0, hi = n_pieces - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (pieces[mid].row_begin <= b) lo = mid;
                else hi = mid - 1;
            }
            s_piece = lo;
        }
        __syncthreads();
        const Piece pc = pieces[s_piece];
        const RowList L = row_list(pc, b, tsel_idx, tsel_cos, stride_t, lsel_idx, lsel_cos, stride_l);
        float *qf = reinterpret_cast<float *>(qs);
        for (int d = tid; d < dim_pad; d += FB_TH) {
            const int64_t o = L.grow * (int64_t)dim_pad + d;
            float x;
            if (q32) {
                x = q32[o];
            } else {
                const __half h = __ushort_as_half(q_hi[o]), l = __ushort_as_half(q_lo[o]);
                x = fmaf(__half2float(l), 1.f / 2048.f, __half2float(h));
            }
            qf[d] = x;
        }
        __syncthreads();
        const int n = pc.n_obj, nv = dim_pad / 4;
        for (int j = tid; j < n; j += FB_TH) {
            const float4 *dj = reinterpret_cast<const float4 *>(pc.d32 + (int64_t)j * dim_pad);
            float acc = 0.f;
            for (int v = 0; v < nv; ++v) {
                const float4 a = qs[v], d = __ldg(dj + v);
                acc = fmaf(a.x, d.x, acc);
                acc = fmaf(a.y, d.y, acc);
                acc = fmaf(a.z, d.z, acc);
                acc = fmaf(a.w, d.w, acc);
            }
            row[j] = acc;
        }
        __syncthreads();
        const int keep = L.keep < n ? L.keep : n;
        sel::select_row_global<FB_TH>(row, n, keep, cand, hist, s_misc, L.oi, L.oc, L.stride, 0.f);
        __syncthreads();
    }
}

}  // namespace

cudaError_t launch_fuse_fallback(const Piece *pieces, int32_t n_pieces, const int32_t *n_overflow,
                                 const int32_t *overflow_rows, const float *q32, const uint16_t *q_hi,
                                 const uint16_t *q_lo, int32_t dim_pad, int32_t *tsel_idx, float *tsel_cos,
                                 int32_t stride_t, int32_t *lsel_idx, float *lsel_cos, int32_t stride_l, float *slab,
                                 int64_t slab_ld, int32_t blocks, int32_t *n_fallback, cudaStream_t st)
{
    if (n_pieces < 1 || blocks < 1 || !n_overflow || !overflow_rows || !slab || dim_pad % 4 != 0 ||
        (!q32 && (!q_hi || !q_lo)) || !tsel_cos || !lsel_cos)
        return cudaErrorInvalidValue;
    const size_t smem = (size_t)dim_pad * sizeof(float);
    if (smem > 48 * 1024) {
        const cudaError_t e =
            cudaFuncSetAttribute(fuse_fallback_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    fuse_fallback_kernel<<<(unsigned)blocks, FB_TH, smem, st>>>(pieces, n_pieces, n_overflow, overflow_rows, q32, q_hi,
                                                              q_lo, dim_pad, tsel_idx, tsel_cos, stride_t, lsel_idx,
                                                              lsel_cos, stride_l, slab, slab_ld, n_fallback);
    return cudaGetLastError();
}

cudaError_t launch_fuse_sample_tau(const float *S, const float *tops, const Piece *pieces, int32_t n_pieces,
                                   int64_t total_rows, const FuseEmit &emit, cudaStream_t st)
{
    if (total_rows <= 0) return cudaSuccess;
    if (n_pieces < 1 || !S || !tops || !emit.tau_key || !emit.cnt || !emit.cand) return cudaErrorInvalidValue;
    const int64_t blocks = (total_rows + TAU_WARPS - 1) / TAU_WARPS;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
    sample_tau_kernel<<<(unsigned)blocks, TAU_WARPS * 32, 0, st>>>(S, tops, pieces, n_pieces, total_rows, emit);
    return cudaGetLastError();
}

cudaError_t launch_fuse_maxima_tau(const float *tops, const Piece *pieces, int32_t n_pieces, int64_t total_rows,
                                   const FuseEmit &emit, int32_t gmax, cudaStream_t st)
{
    if (total_rows <= 0) return cudaSuccess;
    if (n_pieces < 1 || !tops || !emit.tau_key || !emit.cnt || gmax < 1 || gmax > kMaximaTauKeys)
        return cudaErrorInvalidValue;
    const int64_t blocks = (total_rows + TAU_WARPS - 1) / TAU_WARPS;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
    const size_t smem = (size_t)TAU_WARPS * gmax * sizeof(uint32_t);
    if (smem > 48 * 1024) {
        const cudaError_t e =
            cudaFuncSetAttribute(maxima_tau_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    maxima_tau_kernel<<<(unsigned)blocks, TAU_WARPS * 32, smem, st>>>(tops, pieces, n_pieces, total_rows, emit, gmax);
    return cudaGetLastError();
}

int fuse_merge_capacity(int32_t) { return 2048; }

cudaError_t launch_fuse_final(const Piece *pieces, int32_t n_pieces, int64_t total_rows, int32_t *tsel_idx,
                              float *tsel_cos, int32_t stride_t, int32_t *lsel_idx, float *lsel_cos, int32_t stride_l,
                              const FuseEmit &emit, int32_t *n_overflow, int32_t *overflow_rows, int32_t *n_big,
                              int32_t *big_rows, int32_t max_keep, cudaStream_t st)
{
    if (total_rows <= 0) return cudaSuccess;
    if (n_pieces < 1 || !tsel_cos || !lsel_cos || !emit.cnt || !emit.cand || !n_overflow || !overflow_rows ||
        !n_big || !big_rows || max_keep < 1 || max_keep > kMaxTargetCands || emit.cap > 64 * 32)
        return cudaErrorInvalidValue;
    constexpr int FW = 4;
    const int64_t blocks = (total_rows + FW - 1) / FW;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
    fuse_final_kernel<FW><<<(unsigned)blocks, FW * 32, 0, st>>>(pieces, n_pieces, total_rows, tsel_idx, tsel_cos,
                                                                stride_t, lsel_idx, lsel_cos, stride_l, emit,
                                                                n_overflow, overflow_rows, n_big, big_rows);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    fuse_final_big_kernel<64><<<FINAL_BIG_BLOCKS, 32, 0, st>>>(pieces, n_pieces, tsel_idx, tsel_cos, stride_t,
                                                                lsel_idx, lsel_cos, stride_l, emit, n_big, big_rows,
                                                                n_overflow, overflow_rows);
    return cudaGetLastError();
}

}  // namespace farm
