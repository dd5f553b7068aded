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

__global__ void __launch_bounds__(TH)
rescore_kernel(const float *__restrict__ Q32, int64_t q_row0, int32_t dim_pad, const float *__restrict__ D32,
               const int32_t *__restrict__ cand, const float *__restrict__ cand_val, float band, int32_t C,
               int32_t cand_stride, int64_t cand_row0, int32_t R, int32_t *__restrict__ out_idx,
               float *__restrict__ out_cos, int32_t out_stride, int64_t out_row0)
{
    extern __shared__ float4 q4[];
    __shared__ uint64_t key[SORT_MAX];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t r = blockIdx.x;
    const int nv = dim_pad / 4;
    const float4 *src = reinterpret_cast<const float4 *>(Q32 + (q_row0 + r) * (int64_t)dim_pad);
    for (int i = tid; i < nv; i += TH) q4[i] = src[i];
    __syncthreads();
    const int32_t *cr = cand + (cand_row0 + r) * (int64_t)cand_stride;
    const float *cv = cand_val ? cand_val + (cand_row0 + r) * (int64_t)cand_stride : nullptr;
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
    int32_t *oi = out_idx + (out_row0 + r) * (int64_t)out_stride;
    float *oc = out_cos ? out_cos + (out_row0 + r) * (int64_t)out_stride : nullptr;
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

}  // namespace farm
