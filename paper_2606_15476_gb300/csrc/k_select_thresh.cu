// k_select_thresh.cu -- thresholded rank selection over the similarity rows
// of the tensor-core paths (App. D.2 step 3 ranks, step 4 landmark
// candidates): the R largest entries of a row, in rank order.
//
// The similarity kernel's epilogue leaves, per row, the maximum of every
// group of 32 (8 in small scenes) consecutive objects.  Those values are
// entries of the row, so the R-th largest of their union, tau, is at most the
// row's R-th largest value: every entry of rank <= R has a value >= tau, and
// it lies in a group whose maximum is >= tau.  Only those groups (about R of
// them) are read: their entries >= tau are the candidates (the top R, their
// ties, and the few entries between tau and the R-th value when two of the
// top R share a group), and a sort of the candidates by (value desc, index
// asc) gives the exact rank list.  A row whose qualifying groups exceed the
// group list is streamed whole instead; a row whose candidates overflow the
// buffer is selected exactly by the global-memory radix select.
//
// Short rows (at most 2,048 objects) with fewer groups than R are staged whole
// in shared memory; their R-th largest key is found there and the candidates
// are taken from the staged keys.
//
// One CTA of 256 threads per row: the group maxima (at most 8,192 values) are
// staged in shared memory and their R-th largest key found by three radix
// passes.
#include "select_common.cuh"

namespace farm {
namespace {

using namespace sel;

constexpr int TT = 256;
constexpr int CAP = 2048;          // candidate words per row before the exact fallback
constexpr int UNION_MAX = 8192;    // union values staged (a prefix of a longer union is still a subset)
constexpr int GLIST = 2048;        // qualifying groups gathered before the row is streamed whole
constexpr int UNROLL = 4;          // float4 loads in flight per thread

__device__ __forceinline__ void push_cand(uint64_t *cand, int *s_cnt, float x, int32_t j)
{
    const int pos = atomicAdd(s_cnt, 1);
    if (pos < CAP) cand[pos] = cand_word(order_key(x), j);
}

// Entries [j0, n) of the row compared against tau (float4 loads from a
// 16-byte aligned j0, scalar loads for the last n % 4).
__device__ __forceinline__ void stream_tail(const float *__restrict__ row, int j0, int n, float tau, uint64_t *cand,
                                            int *s_cnt)
{
    const int tid = threadIdx.x;
    const int n4 = n >> 2, g4 = j0 >> 2;
    const float4 *row4 = reinterpret_cast<const float4 *>(row);
    for (int g0 = g4; g0 < n4; g0 += TT * UNROLL) {
        float4 v[UNROLL];
#pragma unroll
        for (int u = 0; u < UNROLL; ++u) {
            const int g = g0 + u * TT + tid;
            v[u] = g < n4 ? __ldcs(row4 + g) : make_float4(-1e30f, -1e30f, -1e30f, -1e30f);
        }
#pragma unroll
        for (int u = 0; u < UNROLL; ++u) {
            const int g = g0 + u * TT + tid;
            if (g >= n4) continue;
            const float x[4] = {v[u].x, v[u].y, v[u].z, v[u].w};
#pragma unroll
            for (int c = 0; c < 4; ++c)
                if (x[c] >= tau) push_cand(cand, s_cnt, x[c], 4 * g + c);
        }
    }
    for (int j = max(4 * n4, j0) + tid; j < n; j += TT) {
        const float x = __ldcs(row + j);
        if (x >= tau) push_cand(cand, s_cnt, x, j);
    }
}

// Shared memory of one CTA of the block-level select.
struct ThreshSmem {
    uint32_t *ukeys;        // staged group maxima or a short row (dynamic)
    uint64_t *cand;         // CAP candidate words
    uint32_t *hist;         // radix histogram, then the list of qualifying groups (2048 words)
    uint32_t *wsum, *s3;
    int *s_cnt, *s_ng, *s_misc;
};

// The block-level select of thresholded row b (ends with the row written;
// the caller separates rows by a barrier).
__device__ __forceinline__ void thresh_row(const float *__restrict__ S, const float *__restrict__ tops,
                                           const Piece *__restrict__ pieces, int32_t n_pieces, int64_t b,
                                           int32_t *__restrict__ tsel_idx, float *__restrict__ tsel_cos,
                                           int32_t stride_t, int32_t *__restrict__ lsel_idx,
                                           float *__restrict__ lsel_cos, int32_t stride_l,
                                           int32_t *__restrict__ n_fallback, const ThreshSmem &sm)
{
    uint32_t *ukeys = sm.ukeys, *hist = sm.hist, *wsum = sm.wsum, *s3 = sm.s3;
    uint64_t *cand = sm.cand;
    int &s_cnt = *sm.s_cnt, &s_ng = *sm.s_ng;
    int *s_misc = sm.s_misc;
    static_assert(GLIST <= 2048, "the group list reuses the histogram");

    const int tid = threadIdx.x;
    const Piece pc = pieces[find_piece(pieces, n_pieces, b, [](const Piece &x) { return x.tblock_begin; })];
    const int i = pc.th0 + (int)(b - pc.tblock_begin);
    const bool is_tgt = i < pc.ntr;
    const int R = is_tgt ? pc.keep_t : pc.keep_l;
    int32_t *oi;
    float *oc;
    int stride;
    if (is_tgt) {
        const int64_t o = (pc.t_row0 + i) * (int64_t)stride_t;
        oi = tsel_idx + o;
        oc = tsel_cos ? tsel_cos + o : nullptr;
        stride = stride_t;
    } else {
        const int64_t o = (pc.l_row0 + (i - pc.ntr)) * (int64_t)stride_l;
        oi = lsel_idx + o;
        oc = lsel_cos ? lsel_cos + o : nullptr;
        stride = stride_l;
    }
    const int n = pc.n;
    const float *row = S + pc.s_off + (int64_t)i * pc.ld;
    const int gshift = pc.gshift;
    const int64_t n_groups = group_count(n, gshift);
    const int U = (int)min(n_groups, (int64_t)UNION_MAX);
    if (tid == 0) { s_cnt = 0; s_ng = 0; }

    // tau = key_value(T) is an entry of the row (never -0), and for non-NaN x,
    // x >= tau holds exactly when order_key(x) >= T, so the passes below
    // compare floats and build keys only for the entries they keep.
    if (U >= R) {
        // tau: the R-th largest of the group maxima; then the groups whose
        // maximum reaches it, in any order
        const float *tp = tops + pc.tops_off + (int64_t)i * group_stride(n, gshift);
        for (int j = tid; j < U; j += TT) ukeys[j] = order_key(__ldg(tp + j));
        __syncthreads();
        const uint32_t T = kth_key<TT>(ukeys, U, R, hist, wsum, s3);
        const float tau = key_value(T);
        for (int j = tid; j < U; j += TT) {
            if (ukeys[j] >= T) {
                const int pos = atomicAdd(&s_ng, 1);
                if (pos < GLIST) hist[pos] = (uint32_t)j;
            }
        }
        __syncthreads();
        const int ng = s_ng;
        if (ng <= GLIST) {
            // the qualifying groups, read as float4 slots (a group of 32 is
            // eight slots, of 8 two); group starts are 32-byte aligned and a
            // row holds round_up(n, 32) floats, so a slot never leaves it
            const int sshift = gshift - 2;
            const int smask = (1 << sshift) - 1;
            const int slots = ng << sshift;
            for (int s0 = 0; s0 < slots; s0 += TT * UNROLL) {
                float4 v[UNROLL];
                int j4[UNROLL];
#pragma unroll
                for (int u = 0; u < UNROLL; ++u) {
                    const int sl = s0 + u * TT + tid;
                    j4[u] = sl < slots ? (int)((hist[sl >> sshift] << gshift) + ((sl & smask) << 2)) : n;
                    v[u] = j4[u] < n ? __ldcs(reinterpret_cast<const float4 *>(row + j4[u]))
                                     : make_float4(-1e30f, -1e30f, -1e30f, -1e30f);
                }
#pragma unroll
                for (int u = 0; u < UNROLL; ++u) {
                    if (j4[u] >= n) continue;
                    const float x[4] = {v[u].x, v[u].y, v[u].z, v[u].w};
#pragma unroll
                    for (int c = 0; c < 4; ++c)
                        if (j4[u] + c < n && x[c] >= tau) push_cand(cand, &s_cnt, x[c], j4[u] + c);
                }
            }
            // groups past the staged union (rows of more than 8,192 groups)
            if (n_groups > U) stream_tail(row, U << gshift, n, tau, cand, &s_cnt);
        } else {
            stream_tail(row, 0, n, tau, cand, &s_cnt);
        }
    } else if (n <= kSelectSortAll) {
        // a short row: every entry staged, its R-th largest key found in shared memory
        for (int j = tid; j < n; j += TT) ukeys[j] = order_key(__ldcs(row + j));
        __syncthreads();
        const uint32_t T = kth_key<TT>(ukeys, n, R, hist, wsum, s3);
        for (int j = tid; j < n; j += TT) {
            const uint32_t k = ukeys[j];
            if (k >= T) {
                const int pos = atomicAdd(&s_cnt, 1);
                if (pos < CAP) cand[pos] = cand_word(k, j);
            }
        }
    } else {
        // (the planner sends no such row; every entry is a candidate, and the
        // exact select below stands in when they overflow the buffer)
        __syncthreads();
        stream_tail(row, 0, n, -__int_as_float(0x7f800000), cand, &s_cnt);
    }
    __syncthreads();
    const int cnt = s_cnt;
    // (fewer than R candidates cannot happen with group maxima of this row;
    // the exact select then stands in rather than list unfilled entries)
    if (cnt >= R && cnt <= CAP) {
        int P = 1;
        while (P < cnt) P <<= 1;
        for (int j = cnt + tid; j < P; j += TT) cand[j] = 0ull;
        __syncthreads();
        bitonic_desc<TT>(cand, P);
        write_list<TT>(cand, R, 0, nullptr, oi, oc, stride, 0.f);
    } else {
        if (tid == 0) atomicAdd(n_fallback, 1);
        select_row_global<TT>(row, n, R, cand, hist, s_misc, oi, oc, stride, 0.f);
    }
}

#define THRESH_SMEM                                   \
    extern __shared__ uint32_t ukeys[];               \
    __shared__ uint64_t cand[CAP];                    \
    __shared__ uint32_t hist[2048];                   \
    __shared__ uint32_t wsum[TT / 32];                \
    __shared__ uint32_t s3[3];                        \
    __shared__ int s_cnt, s_ng;                       \
    __shared__ int s_misc[TT / 32 + 3];               \
    const ThreshSmem sm{ukeys, cand, hist, wsum, s3, &s_cnt, &s_ng, s_misc};

// One CTA per thresholded row.
__global__ void __launch_bounds__(TT)
select_thresh_kernel(const float *__restrict__ S, const float *__restrict__ tops, const Piece *__restrict__ pieces,
                     int32_t n_pieces, int32_t *__restrict__ tsel_idx, float *__restrict__ tsel_cos, int32_t stride_t,
                     int32_t *__restrict__ lsel_idx, float *__restrict__ lsel_cos, int32_t stride_l,
                     int32_t *__restrict__ n_fallback)
{
    THRESH_SMEM
    thresh_row(S, tops, pieces, n_pieces, blockIdx.x, tsel_idx, tsel_cos, stride_t, lsel_idx, lsel_cos, stride_l,
               n_fallback, sm);
}

// The rows the warp-level select handed on (row_list[0] of them, listed
// from row_list[1]), a grid-stride loop of CTAs.
__global__ void __launch_bounds__(TT)
select_thresh_list_kernel(const float *__restrict__ S, const float *__restrict__ tops,
                          const Piece *__restrict__ pieces, int32_t n_pieces, int32_t *__restrict__ tsel_idx,
                          float *__restrict__ tsel_cos, int32_t stride_t, int32_t *__restrict__ lsel_idx,
                          float *__restrict__ lsel_cos, int32_t stride_l, int32_t *__restrict__ n_fallback,
                          const int32_t *__restrict__ row_list)
{
    THRESH_SMEM
    const int count = row_list[0];
    for (int k = blockIdx.x; k < count; k += gridDim.x) {
        thresh_row(S, tops, pieces, n_pieces, row_list[1 + k], tsel_idx, tsel_cos, stride_t, lsel_idx, lsel_cos,
                   stride_l, n_fallback, sm);
        __syncthreads();            // the next row reuses the shared arrays
    }
}

// ---------------------------------------------------------------------------
// Warp-level select: one warp per row for the common case -- a list of at
// most WS_R entries, at most 4,096 group maxima keyed as at most 1,024 keys
// (maxima of 1, 2 or 4 consecutive groups; or, for a row with fewer group
// maxima than its list length, at most 1,024 entries, ranked directly) --
// with no block barriers.
// The R-th largest key T is found by a bitwise search (the largest T with
// #{keys >= T} >= R), the groups whose maximum reaches it are gathered, and
// the candidates are ranked by counting (at most 32) or sorted by a warp
// bitonic sort (their words are all distinct).  A row outside these limits,
// or whose groups or candidates overflow the warp's buffers, is appended to
// row_list for the block-level select.
constexpr int WS_R = 256;       // longest list a warp selects (the BF16 path's 256 candidates)
constexpr int WS_KPL = 32;      // keys per lane (1,024 per row)
constexpr int WS_GL = 448;      // qualifying groups per warp
constexpr int WS_CAP = 512;     // candidate words per warp
constexpr int WW = 8;           // warps (rows) per CTA
constexpr int WS_GU = 8;        // float4 loads in flight per lane while gathering the groups
constexpr int WS_GL_NARROW = 320;   // qualifying groups per warp (the small-scene kernel)
constexpr int NARROW_R = 128;       // longest list of the small-scene kernel

// The warp-level select of the rows of small scenes (groups of 8 objects)
// with lists of at most NARROW_R entries: the group maxima themselves as
// keys, the qualifying groups gathered with scalar loads, the candidates
// ranked by counting.  (Measured on the 67-scene batch, whose many small
// scenes' lists of 95 and 16 entries these are: 0.95 ms for the select stage
// against 1.05 ms with the general kernel below taking every row.)  Every
// other row is the general kernel's.
__global__ void __launch_bounds__(WW * 32, 4)
select_warp_small_kernel(const float *__restrict__ S, const float *__restrict__ tops, const Piece *__restrict__ pieces,
                   int32_t n_pieces, int64_t total_rows, int32_t *__restrict__ tsel_idx,
                   float *__restrict__ tsel_cos, int32_t stride_t, int32_t *__restrict__ lsel_idx,
                   float *__restrict__ lsel_cos, int32_t stride_l, int32_t *__restrict__ row_list)
{
    __shared__ uint32_t glist_all[WW][WS_GL_NARROW];
    __shared__ uint64_t cand_all[WW][WS_CAP];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t t = (int64_t)blockIdx.x * WW + warp;
    if (t >= total_rows) return;            // (warp-uniform)
    uint32_t *glist = glist_all[warp];
    uint64_t *cand = cand_all[warp];
    const unsigned FULL = 0xffffffffu;
    const unsigned lt = (1u << lane) - 1u;
    auto hand_on = [&]() {
        if (lane == 0) row_list[1 + atomicAdd(&row_list[0], 1)] = (int32_t)t;
    };
    // the piece of thresholded row t (the last whose tblock_begin <= t)
    int lo = 0, hi = n_pieces - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (pieces[mid].tblock_begin <= t) lo = mid;
        else hi = mid - 1;
    }
    const Piece &pc = pieces[lo];
    const int i = pc.th0 + (int)(t - pc.tblock_begin);
    const bool is_tgt = i < pc.ntr;
    const int R = is_tgt ? pc.keep_t : pc.keep_l;
    const int n = pc.n;
    const int gshift = pc.gshift;
    const int64_t n_groups = group_count(n, gshift);
    // a row with fewer group maxima than R (a short row) ranks its entries
    // themselves: their R-th largest key, then every entry reaching it
    const bool entries = n_groups < R;
    if (gshift != kGroupShiftSmall || R > NARROW_R || (entries ? (int64_t)n : n_groups) > 32 * WS_KPL)
        return;    // the general kernel's row
    const int U = entries ? n : (int)n_groups;
    const int kpl = (U + 31) >> 5;
    const float *row = S + pc.s_off + (int64_t)i * pc.ld;
    const float *tp = tops + pc.tops_off + (int64_t)i * group_stride(n, gshift);
    uint32_t key[WS_KPL];
#pragma unroll
    for (int k = 0; k < WS_KPL; ++k) {
        const int g = lane + 32 * k;
        key[k] = (k < kpl && g < U) ? order_key(entries ? __ldcs(row + g) : __ldg(tp + g)) : 0u;  // 0: no value
    }
    // T: the R-th largest key.  It lies between the smallest and the largest
    // key, so it shares their common leading bits; the search sets the bits
    // below them one at a time (keeping a bit while at least R keys reach
    // it), and stops early once exactly R keys reach the candidate: T is
    // then the smallest of those R.
    uint32_t kmax = 0u, kmin = 0xffffffffu;
#pragma unroll
    for (int k = 0; k < WS_KPL; ++k) {
        if (k < kpl && lane + 32 * k < U) {
            kmax = max(kmax, key[k]);
            kmin = min(kmin, key[k]);
        }
    }
    kmax = __reduce_max_sync(FULL, kmax);
    kmin = __reduce_min_sync(FULL, kmin);
    uint32_t T;
    if (kmax == kmin) {
        T = kmax;
    } else {
        const int hb = 31 - __clz(kmax ^ kmin);
        T = hb == 31 ? 0u : (kmax >> (hb + 1)) << (hb + 1);
        for (int bit = hb; bit >= 0; --bit) {
            const uint32_t c = T | (1u << bit);
            int cnt = 0;
#pragma unroll
            for (int k = 0; k < WS_KPL; ++k) cnt += (k < kpl && key[k] >= c) ? 1 : 0;
            const unsigned tot = __reduce_add_sync(FULL, (unsigned)cnt);
            if (tot == (unsigned)R) {
                uint32_t mn = 0xffffffffu;
#pragma unroll
                for (int k = 0; k < WS_KPL; ++k)
                    if (k < kpl && key[k] >= c) mn = min(mn, key[k]);
                T = __reduce_min_sync(FULL, mn);
                break;
            }
            if (tot > (unsigned)R) T = c;
        }
    }
    int cnt = 0;
    if (entries) {
        // the entries reaching T (the top R and their ties) are the candidates
#pragma unroll
        for (int k = 0; k < WS_KPL; ++k) {
            if (k >= kpl) break;
            const bool q = key[k] >= T;
            const unsigned bal = __ballot_sync(FULL, q);
            if (q) {
                const int pos = cnt + __popc(bal & lt);
                if (pos < WS_CAP) cand[pos] = cand_word(key[k], lane + 32 * k);
            }
            cnt += __popc(bal);
        }
    } else {
        // the groups whose maximum reaches T
        int ng = 0;
#pragma unroll
        for (int k = 0; k < WS_KPL; ++k) {
            if (k >= kpl) break;
            const bool q = key[k] >= T;
            const unsigned bal = __ballot_sync(FULL, q);
            if (q) {
                const int pos = ng + __popc(bal & lt);
                if (pos < WS_GL_NARROW) glist[pos] = (uint32_t)(lane + 32 * k);
            }
            ng += __popc(bal);
        }
        if (ng > WS_GL_NARROW) { hand_on(); return; }
        __syncwarp();
        // their entries >= tau
        const float tau = key_value(T);
        const int gmask = (1 << gshift) - 1;
        const int slots = ng << gshift;
        for (int s0 = 0; s0 < slots; s0 += 32 * 4) {
            float x[4];
            int j[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int sl = s0 + 32 * u + lane;
                j[u] = -1;
                if (sl < slots) {
                    const int jj = (int)((glist[sl >> gshift] << gshift) + (sl & gmask));
                    if (jj < n) j[u] = jj;
                }
                x[u] = j[u] >= 0 ? __ldcs(row + j[u]) : 0.f;
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const bool q = j[u] >= 0 && x[u] >= tau;
                const unsigned bal = __ballot_sync(FULL, q);
                if (q) {
                    const int pos = cnt + __popc(bal & lt);
                    if (pos < WS_CAP) cand[pos] = cand_word(order_key(x[u]), j[u]);
                }
                cnt += __popc(bal);
            }
        }
    }
    if (cnt > WS_CAP || cnt < R) { hand_on(); return; }
    __syncwarp();
    // rank by counting: the words are distinct (distinct positions)
    int32_t *oi;
    float *oc;
    int stride;
    if (is_tgt) {
        const int64_t o = (pc.t_row0 + i) * (int64_t)stride_t;
        oi = tsel_idx + o;
        oc = tsel_cos ? tsel_cos + o : nullptr;
        stride = stride_t;
    } else {
        const int64_t o = (pc.l_row0 + (i - pc.ntr)) * (int64_t)stride_l;
        oi = lsel_idx + o;
        oc = lsel_cos ? lsel_cos + o : nullptr;
        stride = stride_l;
    }
    for (int ci = lane; ci < cnt; ci += 32) {
        const uint64_t w = cand[ci];
        int r = 0;
        for (int k = 0; k < cnt; ++k) r += cand[k] > w ? 1 : 0;
        if (r < R) {
            oi[r] = (int32_t)(0xffffffffu - (uint32_t)(w & 0xffffffffu));
            if (oc) oc[r] = key_value((uint32_t)(w >> 32));
        }
    }
    for (int k = R + lane; k < stride; k += 32) {
        oi[k] = -1;
        if (oc) oc[k] = 0.f;
    }
}


// Descending bitonic sort of P words (a power of two, at least 2) by one
// warp, each lane taking compare-exchange pairs (a, a + j) of every stage.
__device__ __forceinline__ void warp_bitonic_desc(uint64_t *w, int P, int lane)
{
    for (int k = 2; k <= P; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int p = lane; p < (P >> 1); p += 32) {
                const int a = ((p & ~(j - 1)) << 1) | (p & (j - 1));
                const uint64_t x = w[a], y = w[a + j];
                const bool desc = (a & k) == 0;
                if (desc ? (x < y) : (x > y)) {
                    w[a] = y;
                    w[a + j] = x;
                }
            }
            __syncwarp();
        }
    }
}

__global__ void __launch_bounds__(WW * 32, 4)
select_warp_kernel(const float *__restrict__ S, const float *__restrict__ tops, const Piece *__restrict__ pieces,
                   int32_t n_pieces, int64_t total_rows, int32_t *__restrict__ tsel_idx,
                   float *__restrict__ tsel_cos, int32_t stride_t, int32_t *__restrict__ lsel_idx,
                   float *__restrict__ lsel_cos, int32_t stride_l, int32_t *__restrict__ row_list)
{
    __shared__ uint32_t glist_all[WW][WS_GL];
    __shared__ uint64_t cand_all[WW][WS_CAP];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t t = (int64_t)blockIdx.x * WW + warp;
    if (t >= total_rows) return;            // (warp-uniform)
    uint32_t *glist = glist_all[warp];
    uint64_t *cand = cand_all[warp];
    const unsigned FULL = 0xffffffffu;
    const unsigned lt = (1u << lane) - 1u;
    auto hand_on = [&]() {
        if (lane == 0) row_list[1 + atomicAdd(&row_list[0], 1)] = (int32_t)t;
    };
    // the piece of thresholded row t (the last whose tblock_begin <= t)
    int lo = 0, hi = n_pieces - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (pieces[mid].tblock_begin <= t) lo = mid;
        else hi = mid - 1;
    }
    const Piece &pc = pieces[lo];
    const int i = pc.th0 + (int)(t - pc.tblock_begin);
    const bool is_tgt = i < pc.ntr;
    const int R = is_tgt ? pc.keep_t : pc.keep_l;
    const int n = pc.n;
    const int gshift = pc.gshift;
    const int64_t n_groups = group_count(n, gshift);
    // a row with fewer group maxima than R (a short row) ranks its entries
    // themselves: their R-th largest key, then every entry reaching it
    const bool entries = n_groups < R;
    if (gshift == kGroupShiftSmall && R <= NARROW_R && (entries ? (int64_t)n : n_groups) <= 32 * WS_KPL)
        return;    // the small-scene kernel's row
    // a row of more than 1,024 group maxima keys the maxima of 2 or 4
    // consecutive groups instead (super-groups: entries of the row too, one
    // per super-group, so their R-th largest still bounds the row's from below)
    int sgs = 0;
    if (!entries)
        while (sgs < 2 && ((n_groups + (1 << sgs) - 1) >> sgs) > 32 * WS_KPL) ++sgs;
    const int64_t n_keys = entries ? (int64_t)n : (n_groups + (1 << sgs) - 1) >> sgs;
    if (R > WS_R || n_keys > 32 * WS_KPL || n_keys < R) { hand_on(); return; }
    const int U = (int)n_keys;
    const int kpl = (U + 31) >> 5;
    const float *row = S + pc.s_off + (int64_t)i * pc.ld;
    // (a row of maxima is 16-byte aligned and holds whole tiles' groups, -inf
    // past the row end, so the 2- and 4-wide loads stay inside it)
    const float *tp = tops + pc.tops_off + (int64_t)i * group_stride(n, gshift);
    uint32_t key[WS_KPL];
#pragma unroll
    for (int k = 0; k < WS_KPL; ++k) {
        const int g = lane + 32 * k;
        uint32_t kk = 0u;   // 0: no value
        if (k < kpl && g < U) {
            if (entries) {
                kk = order_key(__ldcs(row + g));
            } else if (sgs == 0) {
                kk = order_key(__ldg(tp + g));
            } else if (sgs == 1) {
                const float2 v = __ldg(reinterpret_cast<const float2 *>(tp) + g);
                kk = order_key(fmaxf(v.x, v.y));
            } else {
                const float4 v = __ldg(reinterpret_cast<const float4 *>(tp) + g);
                kk = order_key(fmaxf(fmaxf(v.x, v.y), fmaxf(v.z, v.w)));
            }
        }
        key[k] = kk;
    }
    // T: the R-th largest key.  It lies between the smallest and the largest
    // key, so it shares their common leading bits; the search sets the bits
    // below them one at a time (keeping a bit while at least R keys reach
    // it), and stops early once exactly R keys reach the candidate: T is
    // then the smallest of those R.
    uint32_t kmax = 0u, kmin = 0xffffffffu;
#pragma unroll
    for (int k = 0; k < WS_KPL; ++k) {
        if (k < kpl && lane + 32 * k < U) {
            kmax = max(kmax, key[k]);
            kmin = min(kmin, key[k]);
        }
    }
    kmax = __reduce_max_sync(FULL, kmax);
    kmin = __reduce_min_sync(FULL, kmin);
    uint32_t T;
    if (kmax == kmin) {
        T = kmax;
    } else {
        const int hb = 31 - __clz(kmax ^ kmin);
        T = hb == 31 ? 0u : (kmax >> (hb + 1)) << (hb + 1);
        for (int bit = hb; bit >= 0; --bit) {
            const uint32_t c = T | (1u << bit);
            int cnt = 0;
#pragma unroll
            for (int k = 0; k < WS_KPL; ++k) cnt += (k < kpl && key[k] >= c) ? 1 : 0;
            const unsigned tot = __reduce_add_sync(FULL, (unsigned)cnt);
            if (tot == (unsigned)R) {
                uint32_t mn = 0xffffffffu;
#pragma unroll
                for (int k = 0; k < WS_KPL; ++k)
                    if (k < kpl && key[k] >= c) mn = min(mn, key[k]);
                T = __reduce_min_sync(FULL, mn);
                break;
            }
            if (tot > (unsigned)R) T = c;
        }
    }
    int cnt = 0;
    if (entries) {
        // the entries reaching T (the top R and their ties) are the candidates
#pragma unroll
        for (int k = 0; k < WS_KPL; ++k) {
            if (k >= kpl) break;
            const bool q = key[k] >= T;
            const unsigned bal = __ballot_sync(FULL, q);
            if (q) {
                const int pos = cnt + __popc(bal & lt);
                if (pos < WS_CAP) cand[pos] = cand_word(key[k], lane + 32 * k);
            }
            cnt += __popc(bal);
        }
    } else {
        // the groups whose maximum reaches T (those of the super-groups whose
        // maximum does)
        const float tau = key_value(T);
        int ng = 0;
#pragma unroll
        for (int k = 0; k < WS_KPL; ++k) {
            if (k >= kpl) break;
            const bool qs = key[k] >= T;
            if (sgs == 0) {
                const unsigned bal = __ballot_sync(FULL, qs);
                if (qs) {
                    const int pos = ng + __popc(bal & lt);
                    if (pos < WS_GL) glist[pos] = (uint32_t)(lane + 32 * k);
                }
                ng += __popc(bal);
            } else if (__any_sync(FULL, qs)) {
                for (int c = 0; c < (1 << sgs); ++c) {
                    const int g = ((lane + 32 * k) << sgs) + c;
                    const bool q = qs && g < n_groups && __ldg(tp + g) >= tau;
                    const unsigned bal = __ballot_sync(FULL, q);
                    if (q) {
                        const int pos = ng + __popc(bal & lt);
                        if (pos < WS_GL) glist[pos] = (uint32_t)g;
                    }
                    ng += __popc(bal);
                }
            }
        }
        if (ng > WS_GL) { hand_on(); return; }
        __syncwarp();
        // their entries >= tau, read as float4 slots (a group of 32 is eight
        // slots, of 8 two; group starts are 32-byte aligned and a row holds
        // round_up(n, 32) floats, so a slot never leaves it), WS_GU slots in
        // flight per lane
        const int sshift = gshift - 2;
        const int smask = (1 << sshift) - 1;
        const int slots = ng << sshift;
        for (int s0 = 0; s0 < slots; s0 += 32 * WS_GU) {
            float4 v[WS_GU];
            int j4[WS_GU];
#pragma unroll
            for (int u = 0; u < WS_GU; ++u) {
                const int sl = s0 + 32 * u + lane;
                j4[u] = sl < slots ? (int)((glist[sl >> sshift] << gshift) + ((sl & smask) << 2)) : n;
                v[u] = j4[u] < n ? __ldcs(reinterpret_cast<const float4 *>(row + j4[u])) : make_float4(0.f, 0.f, 0.f, 0.f);
            }
#pragma unroll
            for (int u = 0; u < WS_GU; ++u) {
                if (s0 + 32 * u >= slots) break;     // (warp-uniform: short lists take few ballots)
                const float x[4] = {v[u].x, v[u].y, v[u].z, v[u].w};
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const bool q = j4[u] + c < n && x[c] >= tau;
                    const unsigned bal = __ballot_sync(FULL, q);
                    if (q) {
                        const int pos = cnt + __popc(bal & lt);
                        if (pos < WS_CAP) cand[pos] = cand_word(order_key(x[c]), j4[u] + c);
                    }
                    cnt += __popc(bal);
                }
            }
        }
    }
    if (cnt > WS_CAP || cnt < R) { hand_on(); return; }
    // order the candidate words (distinct: distinct positions): at most 32
    // are ranked by counting, more sorted by a bitonic sort (padded with zero
    // words to a power of two), in descending order
    __syncwarp();
    if (cnt <= 32) {
        const uint64_t w = lane < cnt ? cand[lane] : 0ull;
        int r = 0;
        for (int k = 0; k < cnt; ++k) r += cand[k] > w ? 1 : 0;
        __syncwarp();
        if (lane < cnt) cand[r] = w;
        __syncwarp();
    } else {
        int P = 64;
        while (P < cnt) P <<= 1;
        for (int k = cnt + lane; k < P; k += 32) cand[k] = 0ull;
        __syncwarp();
        warp_bitonic_desc(cand, P, lane);
    }
    int32_t *oi;
    float *oc;
    int stride;
    if (is_tgt) {
        const int64_t o = (pc.t_row0 + i) * (int64_t)stride_t;
        oi = tsel_idx + o;
        oc = tsel_cos ? tsel_cos + o : nullptr;
        stride = stride_t;
    } else {
        const int64_t o = (pc.l_row0 + (i - pc.ntr)) * (int64_t)stride_l;
        oi = lsel_idx + o;
        oc = lsel_cos ? lsel_cos + o : nullptr;
        stride = stride_l;
    }
    for (int r = lane; r < R; r += 32) {
        const uint64_t w = cand[r];
        oi[r] = (int32_t)(0xffffffffu - (uint32_t)(w & 0xffffffffu));
        if (oc) oc[r] = key_value((uint32_t)(w >> 32));
    }
    for (int k = R + lane; k < stride; k += 32) {
        oi[k] = -1;
        if (oc) oc[k] = 0.f;
    }
}

}  // namespace

cudaError_t launch_select_thresh(const float *S, const float *tops, const Piece *pieces, int32_t n_pieces,
                                 int64_t total_blocks, int32_t max_union, int32_t *tsel_idx, float *tsel_cos,
                                 int32_t stride_t, int32_t *lsel_idx, float *lsel_cos, int32_t stride_l,
                                 int32_t *n_fallback, int32_t *row_list, cudaStream_t s)
{
    if (total_blocks <= 0) return cudaSuccess;
    if (n_pieces < 1 || total_blocks > 0x7fffffff || max_union < 1 || ((uintptr_t)S & 15u) != 0 ||
        ((uintptr_t)tops & 15u) != 0 || !n_fallback)
        return cudaErrorInvalidValue;
    // the staged group maxima, or a whole short row
    const int32_t staged = max_union < UNION_MAX ? (max_union > kSelectSortAll ? max_union : kSelectSortAll) : UNION_MAX;
    const size_t smem = (size_t)staged * sizeof(uint32_t);
    static_assert(CAP >= kSelectSortAll, "rows that take every entry fit the candidate buffer");
    cudaError_t e;
    if (!row_list) {
        e = cudaFuncSetAttribute(select_thresh_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        select_thresh_kernel<<<(unsigned)total_blocks, TT, smem, s>>>(S, tops, pieces, n_pieces, tsel_idx, tsel_cos,
                                                                      stride_t, lsel_idx, lsel_cos, stride_l,
                                                                      n_fallback);
        return cudaGetLastError();
    }
    // the warp-level selects first (each takes its own rows); the rows they
    // hand on go to the block-level one
    if ((e = cudaMemsetAsync(row_list, 0, sizeof(int32_t), s)) != cudaSuccess) return e;
    select_warp_small_kernel<<<(unsigned)((total_blocks + WW - 1) / WW), WW * 32, 0, s>>>(
        S, tops, pieces, n_pieces, total_blocks, tsel_idx, tsel_cos, stride_t, lsel_idx, lsel_cos, stride_l, row_list);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    select_warp_kernel<<<(unsigned)((total_blocks + WW - 1) / WW), WW * 32, 0, s>>>(
        S, tops, pieces, n_pieces, total_blocks, tsel_idx, tsel_cos, stride_t, lsel_idx, lsel_cos, stride_l, row_list);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    e = cudaFuncSetAttribute(select_thresh_list_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int64_t grid = total_blocks < 2048 ? total_blocks : 2048;
    select_thresh_list_kernel<<<(unsigned)grid, TT, smem, s>>>(S, tops, pieces, n_pieces, tsel_idx, tsel_cos,
                                                               stride_t, lsel_idx, lsel_cos, stride_l, n_fallback,
                                                               row_list);
    return cudaGetLastError();
}

}  // namespace farm
