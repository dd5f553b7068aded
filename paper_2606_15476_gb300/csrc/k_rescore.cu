// k_rescore.cu -- FP32 re-scoring of the reduced-precision path's candidates.
//
// The BF16 similarity stage ranks every object approximately; for each row
// its C best objects are then re-scored with exact FP32 dot products of the
// unit rows (App. D.2 step 3 cosines) and the R best of them, in rank order
// (cosine descending, lower index first), become the row's rank list.  The
// result equals the FP32 path's list whenever the FP32 top R lie within the
// BF16 top C.
//
// Only the borderline candidates are re-scored: with the reduced-precision
// values of the (descending) candidate list at hand, a candidate whose value
// lies more than `band` below the R-th value is skipped (it would need an
// arithmetic error above the band to belong to the top R).
//
// Rows of a scene that ran the FP32-accurate similarity in the same batch
// (Piece::exact) already hold their final lists: copy_lists_kernel copies
// them, a warp per row.
//
// One CTA per row: the row is staged in shared memory, each warp takes two
// candidates at a time (lanes stride both descriptors in float4 with four
// loads of each in flight, then shuffle reductions), and a bitonic sort over
// (cosine key, index) orders the scores.
#include "farm_internal.h"

namespace farm {
namespace {

constexpr int TH = 256;
constexpr int SORT_MAX = 1024;

__device__ __forceinline__ uint32_t order_key(float f)
{
    const uint32_t u = __float_as_uint(f + 0.0f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

__device__ __forceinline__ float key_value(uint32_t k)
{
    const uint32_t u = (k & 0x80000000u) ? (k & 0x7fffffffu) : ~k;
    return __uint_as_float(u);
}

// One row: the C candidates cr (values cv, nullable) against the unit row q
// (global, dim_pad floats) -> the R best in rank order into oi / oc.
__device__ __forceinline__ void rescore_row(const float *__restrict__ q, int32_t dim_pad,
                                            const float *__restrict__ D32, const int32_t *__restrict__ cr,
                                            const float *__restrict__ cv, float band, int32_t C, int32_t R,
                                            int32_t *__restrict__ oi, float *__restrict__ oc, int32_t out_stride)
{
    extern __shared__ float4 q4[];
    __shared__ uint64_t key[SORT_MAX];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nv = dim_pad / 4;
    const float4 *src = reinterpret_cast<const float4 *>(q);
    for (int i = tid; i < nv; i += TH) q4[i] = src[i];
    __syncthreads();
    const float thr = cv ? cv[R - 1] - band : 0.f;
    // two candidates per warp step, four float4 loads of each in flight per lane
    for (int c0 = 2 * warp; c0 < C; c0 += 2 * (TH / 32)) {
        const int c1 = c0 + 1;
        const bool do0 = !(cv && cv[c0] < thr);
        const bool do1 = c1 < C && !(cv && cv[c1] < thr);
        if (!do0 && !do1) {
            if (lane == 0) {
                key[c0] = 0ull;
                if (c1 < C) key[c1] = 0ull;
            }
            continue;
        }
        const int32_t e0 = do0 ? cr[c0] : 0, e1 = do1 ? cr[c1] : 0;
        const float4 *p0 = reinterpret_cast<const float4 *>(D32 + (int64_t)e0 * dim_pad);
        const float4 *p1 = reinterpret_cast<const float4 *>(D32 + (int64_t)e1 * dim_pad);
        float a0 = 0.f, a1 = 0.f;
        for (int base = 0; base < nv; base += 4 * 32) {
            float4 x0[4], x1[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int i = base + u * 32 + lane;
                const bool in = i < nv;
                x0[u] = (in && do0) ? __ldg(p0 + i) : make_float4(0.f, 0.f, 0.f, 0.f);
                x1[u] = (in && do1) ? __ldg(p1 + i) : make_float4(0.f, 0.f, 0.f, 0.f);
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int i = base + u * 32 + lane;
                if (i < nv) {
                    const float4 q = q4[i];
                    a0 = fmaf(q.x, x0[u].x, a0);
                    a0 = fmaf(q.y, x0[u].y, a0);
                    a0 = fmaf(q.z, x0[u].z, a0);
                    a0 = fmaf(q.w, x0[u].w, a0);
                    a1 = fmaf(q.x, x1[u].x, a1);
                    a1 = fmaf(q.y, x1[u].y, a1);
                    a1 = fmaf(q.z, x1[u].z, a1);
                    a1 = fmaf(q.w, x1[u].w, a1);
                }
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            a0 += __shfl_xor_sync(0xffffffffu, a0, o);
            a1 += __shfl_xor_sync(0xffffffffu, a1, o);
        }
        if (lane == 0) {
            key[c0] = do0 ? ((uint64_t)order_key(a0) << 32) | (uint64_t)(0xffffffffu - (uint32_t)e0) : 0ull;
            if (c1 < C) key[c1] = do1 ? ((uint64_t)order_key(a1) << 32) | (uint64_t)(0xffffffffu - (uint32_t)e1) : 0ull;
        }
    }
    int P = 1;
    while (P < C) P <<= 1;
    for (int i = C + tid; i < P; i += TH) key[i] = 0ull;
    __syncthreads();
    for (int k = 2; k <= P; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = tid; i < P; i += TH) {
                const int ixj = i ^ j;
                if (ixj > i) {
                    const uint64_t a = key[i], b = key[ixj];
                    const bool desc = (i & k) == 0;
                    if (desc ? (a < b) : (a > b)) { key[i] = b; key[ixj] = a; }
                }
            }
            __syncthreads();
        }
    }
    for (int i = tid; i < out_stride; i += TH) {
        if (i < R) {
            oi[i] = (int32_t)(0xffffffffu - (uint32_t)(key[i] & 0xffffffffu));
            if (oc) oc[i] = key_value((uint32_t)(key[i] >> 32));
        } else {
            oi[i] = -1;
            if (oc) oc[i] = 0.f;
        }
    }
}

// Grouped rescore: block -> (piece, row) through the piece table.
__global__ void __launch_bounds__(TH)
rescore_grouped_kernel(const Piece *__restrict__ pieces, int32_t n_pieces, const float *__restrict__ Q32,
                       int32_t dim_pad, const int32_t *__restrict__ bsel_t, const float *__restrict__ bsel_tv,
                       int32_t cstride_t, const int32_t *__restrict__ bsel_l, const float *__restrict__ bsel_lv,
                       int32_t cstride_l, float band, int32_t *__restrict__ tsel_idx, float *__restrict__ tsel_cos,
                       int32_t stride_t, int32_t *__restrict__ lsel_idx, int32_t stride_l)
{
    const int64_t r = blockIdx.x;
    const Piece pc = pieces[find_piece(pieces, n_pieces, r, [](const Piece &x) { return x.row_begin; })];
    const int i = (int)(r - pc.row_begin);
    const float *q = Q32 + (pc.q_row0 + i) * (int64_t)dim_pad;
    if (i < pc.ntr) {
        const int64_t co = (pc.t_row0 + i) * (int64_t)cstride_t, oo = (pc.t_row0 + i) * (int64_t)stride_t;
        rescore_row(q, dim_pad, pc.d32, bsel_t + co, bsel_tv ? bsel_tv + co : nullptr, band, pc.fkeep_t, pc.R,
                    tsel_idx + oo, tsel_cos ? tsel_cos + oo : nullptr, stride_t);
    } else {
        const int64_t l = pc.l_row0 + (i - pc.ntr);
        const int64_t co = l * (int64_t)cstride_l;
        rescore_row(q, dim_pad, pc.d32, bsel_l + co, bsel_lv ? bsel_lv + co : nullptr, band, pc.fkeep_l, pc.klm,
                    lsel_idx + l * (int64_t)stride_l, nullptr, stride_l);
    }
}

// The final lists of launch rows [row0, row0 + rows) -- rows of FP32-accurate
// scenes -- copied from the candidate buffers: R (klm) entries, -1 / 0 past them.
__global__ void __launch_bounds__(256)
copy_lists_kernel(const Piece *__restrict__ pieces, int32_t n_pieces, int64_t row0, int64_t rows,
                  const int32_t *__restrict__ bsel_t, const float *__restrict__ bsel_tv, int32_t cstride_t,
                  const int32_t *__restrict__ bsel_l, int32_t cstride_l, int32_t *__restrict__ tsel_idx,
                  float *__restrict__ tsel_cos, int32_t stride_t, int32_t *__restrict__ lsel_idx, int32_t stride_l)
{
    const int lane = threadIdx.x & 31;
    const int64_t w = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
    if (w >= rows) return;
    const int64_t r = row0 + w;
    int lo = 0;
    if (lane == 0) {
        int hi = n_pieces - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (pieces[mid].row_begin <= r) lo = mid;
            else hi = mid - 1;
        }
    }
    const Piece &pc = pieces[__shfl_sync(0xffffffffu, lo, 0)];
    const int i = (int)(r - pc.row_begin);
    const bool tgt = i < pc.ntr;
    const int64_t l = pc.l_row0 + (i - pc.ntr);
    const int64_t co = tgt ? (pc.t_row0 + i) * (int64_t)cstride_t : l * (int64_t)cstride_l;
    const int32_t *src = (tgt ? bsel_t : bsel_l) + co;
    int32_t *oi = tgt ? tsel_idx + (pc.t_row0 + i) * (int64_t)stride_t : lsel_idx + l * (int64_t)stride_l;
    float *oc = tgt && tsel_cos ? tsel_cos + (pc.t_row0 + i) * (int64_t)stride_t : nullptr;
    const int keep = tgt ? pc.R : pc.klm, out = tgt ? stride_t : stride_l;
    for (int k = lane; k < out; k += 32) {
        oi[k] = k < keep ? src[k] : -1;
        if (oc) oc[k] = k < keep ? bsel_tv[co + k] : 0.f;
    }
}

}  // namespace

cudaError_t launch_copy_lists(const Piece *pieces, int32_t n_pieces, int64_t row0, int64_t rows, const int32_t *bsel_t,
                              const float *bsel_tv, int32_t cstride_t, const int32_t *bsel_l, int32_t cstride_l,
                              int32_t *tsel_idx, float *tsel_cos, int32_t stride_t, int32_t *lsel_idx,
                              int32_t stride_l, cudaStream_t s)
{
    if (rows <= 0) return cudaSuccess;
    if (n_pieces < 1 || (tsel_cos && !bsel_tv)) return cudaErrorInvalidValue;
    const int64_t blocks = (rows + 7) / 8;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
    copy_lists_kernel<<<(unsigned)blocks, 256, 0, s>>>(pieces, n_pieces, row0, rows, bsel_t, bsel_tv, cstride_t,
                                                        bsel_l, cstride_l, tsel_idx, tsel_cos, stride_t, lsel_idx,
                                                        stride_l);
    return cudaGetLastError();
}

cudaError_t launch_rescore_grouped(const Piece *pieces, int32_t n_pieces, int64_t total_rows, const float *Q32,
                                   int32_t dim_pad, const int32_t *bsel_t, const float *bsel_tv, int32_t cstride_t,
                                   const int32_t *bsel_l, const float *bsel_lv, int32_t cstride_l, float band,
                                   int32_t *tsel_idx, float *tsel_cos, int32_t stride_t, int32_t *lsel_idx,
                                   int32_t stride_l, cudaStream_t s)
{
    if (total_rows <= 0) return cudaSuccess;
    if (n_pieces < 1 || total_rows > 0x7fffffff || dim_pad % 4 != 0 || cstride_t > SORT_MAX || cstride_l > SORT_MAX)
        return cudaErrorInvalidValue;
    const size_t smem = (size_t)dim_pad * sizeof(float);
    if (smem > 48 * 1024) {
        cudaError_t e =
            cudaFuncSetAttribute(rescore_grouped_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    rescore_grouped_kernel<<<(unsigned)total_rows, TH, smem, s>>>(pieces, n_pieces, Q32, dim_pad, bsel_t, bsel_tv,
                                                                  cstride_t, bsel_l, bsel_lv, cstride_l, band,
                                                                  tsel_idx, tsel_cos, stride_t, lsel_idx, stride_l);
    return cudaGetLastError();
}

}  // namespace farm
