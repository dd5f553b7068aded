// k_select_thresh.cu -- thresholded rank selection over the similarity rows
// of the tensor-core paths (App. D.2 step 3 ranks, step 4 landmark
// candidates): the R largest entries of a row, in rank order.
//
// The similarity kernel's epilogue leaves, per row, the maximum of every
// group of 32 (8 in small scenes) consecutive objects.  Those values are entries of the row, so
// the R-th largest of their union, tau, is at most the row's R-th largest
// value: every entry of rank <= R has a value >= tau.  One pass over the row
// collects the entries >= tau (the top R, their ties, and the few entries
// between tau and the R-th value when two of the top R share a group), and a
// sort of those candidates by (value desc, index asc) gives the exact rank
// list.  A row whose candidates overflow the buffer is
// selected exactly by the global-memory radix select instead.
//
// One CTA of 256 threads per row: the union (at most 8,192 values) is staged
// in shared memory and its R-th largest key found by three radix passes;
// the row is streamed once from global memory with evict-first loads.
#include "select_common.cuh"

namespace farm {
namespace {

using namespace sel;

constexpr int TT = 256;
constexpr int CAP = 2048;          // candidate words per row before the exact fallback
constexpr int UNION_MAX = 8192;    // union values staged (a prefix of a longer union is still a subset)
constexpr int UNROLL = 4;          // float4 loads in flight per thread

__global__ void __launch_bounds__(TT)
select_thresh_kernel(const float *__restrict__ S, const float *__restrict__ tops, const Piece *__restrict__ pieces,
                     int32_t n_pieces, int32_t *__restrict__ tsel_idx, float *__restrict__ tsel_cos, int32_t stride_t,
                     int32_t *__restrict__ lsel_idx, float *__restrict__ lsel_cos, int32_t stride_l,
                     int32_t *__restrict__ n_fallback)
{
    extern __shared__ uint32_t ukeys[];
    __shared__ uint64_t cand[CAP];
    __shared__ uint32_t hist[2048];
    __shared__ uint32_t wsum[TT / 32];
    __shared__ uint32_t s3[3];
    __shared__ int s_cnt;
    __shared__ int s_misc[TT / 32 + 3];

    const int tid = threadIdx.x;
    const int64_t b = blockIdx.x;
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
    const int U = (int)min(group_count(n, pc.gshift), (int64_t)UNION_MAX);

    // tau: the R-th largest of the group maxima; a row with fewer groups than
    // R (the planner sends only rows of at most kSelectSortAll objects) takes
    // every entry as a candidate.  tau = key_value(T) is the group value
    // itself (never -0), and for non-NaN x, x >= tau holds exactly when
    // order_key(x) >= T, so the pass below compares floats and builds keys
    // only for the entries it keeps.
    float tau = -__int_as_float(0x7f800000);
    if (U >= R) {
        const float *tp = tops + pc.tops_off + (int64_t)i * group_stride(n, pc.gshift);
        for (int j = tid; j < U; j += TT) ukeys[j] = order_key(__ldg(tp + j));
        __syncthreads();
        tau = key_value(kth_key<TT>(ukeys, U, R, hist, wsum, s3));
    }
    if (tid == 0) s_cnt = 0;
    __syncthreads();
    const int n4 = n >> 2;
    const float4 *row4 = reinterpret_cast<const float4 *>(row);
    for (int g0 = 0; g0 < n4; g0 += TT * UNROLL) {
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
            for (int c = 0; c < 4; ++c) {
                if (x[c] >= tau) {
                    const int pos = atomicAdd(&s_cnt, 1);
                    if (pos < CAP) cand[pos] = cand_word(order_key(x[c]), 4 * g + c);
                }
            }
        }
    }
    for (int j = 4 * n4 + tid; j < n; j += TT) {
        const float x = __ldcs(row + j);
        if (x >= tau) {
            const int pos = atomicAdd(&s_cnt, 1);
            if (pos < CAP) cand[pos] = cand_word(order_key(x), j);
        }
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

}  // namespace

cudaError_t launch_select_thresh(const float *S, const float *tops, const Piece *pieces, int32_t n_pieces,
                                 int64_t total_blocks, int32_t max_union, int32_t *tsel_idx, float *tsel_cos,
                                 int32_t stride_t, int32_t *lsel_idx, float *lsel_cos, int32_t stride_l,
                                 int32_t *n_fallback, cudaStream_t s)
{
    if (total_blocks <= 0) return cudaSuccess;
    if (n_pieces < 1 || total_blocks > 0x7fffffff || max_union < 1 || ((uintptr_t)S & 15u) != 0 ||
        ((uintptr_t)tops & 15u) != 0 || !n_fallback)
        return cudaErrorInvalidValue;
    const size_t smem = (size_t)(max_union < UNION_MAX ? max_union : UNION_MAX) * sizeof(uint32_t);
    static_assert(CAP >= kSelectSortAll, "rows that take every entry fit the candidate buffer");
    cudaError_t e = cudaFuncSetAttribute(select_thresh_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    select_thresh_kernel<<<(unsigned)total_blocks, TT, smem, s>>>(S, tops, pieces, n_pieces, tsel_idx, tsel_cos,
                                                                  stride_t, lsel_idx, lsel_cos, stride_l, n_fallback);
    return cudaGetLastError();
}

}  // namespace farm
