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
// One CTA per row: the row is staged in shared memory, each warp takes
// candidates in turn (lanes stride the descriptor in float4, then a shuffle
// reduction), and a bitonic sort over (cosine key, index) orders the scores.
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
    for (int c = warp; c < C; c += TH / 32) {
        if (cv && cv[c] < thr) {
            if (lane == 0) key[c] = 0ull;
            continue;
        }
        const int32_t e = cr[c];
        const float4 *dp = reinterpret_cast<const float4 *>(D32 + (int64_t)e * dim_pad);
        float acc = 0.f;
        for (int i = lane; i < nv; i += 32) {
            const float4 a = q4[i], b = __ldg(dp + i);
            acc = fmaf(a.x, b.x, acc);
            acc = fmaf(a.y, b.y, acc);
            acc = fmaf(a.z, b.z, acc);
            acc = fmaf(a.w, b.w, acc);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) key[c] = ((uint64_t)order_key(acc) << 32) | (uint64_t)(0xffffffffu - (uint32_t)e);
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

__global__ void __launch_bounds__(TH)
rescore_kernel(const float *__restrict__ Q32, int64_t q_row0, int32_t dim_pad, const float *__restrict__ D32,
               const int32_t *__restrict__ cand, const float *__restrict__ cand_val, float band, int32_t C,
               int32_t cand_stride, int64_t cand_row0, int32_t R, int32_t *__restrict__ out_idx,
               float *__restrict__ out_cos, int32_t out_stride, int64_t out_row0)
{
    const int64_t r = blockIdx.x;
    const int64_t co = (cand_row0 + r) * (int64_t)cand_stride, oo = (out_row0 + r) * (int64_t)out_stride;
    rescore_row(Q32 + (q_row0 + r) * (int64_t)dim_pad, dim_pad, D32, cand + co, cand_val ? cand_val + co : nullptr,
                band, C, R, out_idx + oo, out_cos ? out_cos + oo : nullptr, out_stride);
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
        rescore_row(q, dim_pad, pc.d32, bsel_t + co, bsel_tv ? bsel_tv + co : nullptr, band, pc.keep_t, pc.R,
                    tsel_idx + oo, tsel_cos ? tsel_cos + oo : nullptr, stride_t);
    } else {
        const int64_t l = pc.l_row0 + (i - pc.ntr);
        const int64_t co = l * (int64_t)cstride_l;
        rescore_row(q, dim_pad, pc.d32, bsel_l + co, bsel_lv ? bsel_lv + co : nullptr, band, pc.keep_l, pc.klm,
                    lsel_idx + l * (int64_t)stride_l, nullptr, stride_l);
    }
}

}  // namespace

cudaError_t launch_rescore(const float *Q32, int64_t q_row0, int32_t dim_pad, const float *D32, const int32_t *cand,
                           const float *cand_val, float band, int32_t C, int32_t cand_stride, int64_t cand_row0,
                           int64_t rows, int32_t R, int32_t *out_idx, float *out_cos, int32_t out_stride,
                           int64_t out_row0, cudaStream_t s)
{
    if (rows <= 0) return cudaSuccess;
    if (C < 1 || C > SORT_MAX || R < 1 || R > C || R > out_stride || dim_pad % 4 != 0) return cudaErrorInvalidValue;
    const size_t smem = (size_t)dim_pad * sizeof(float);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(rescore_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    rescore_kernel<<<(unsigned)rows, TH, smem, s>>>(Q32, q_row0, dim_pad, D32, cand, cand_val, band, C, cand_stride,
                                                    cand_row0, R, out_idx, out_cos, out_stride, out_row0);
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
