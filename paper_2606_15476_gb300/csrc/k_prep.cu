// k_prep.cu -- row normalisation, operand splits and per-view records.
//
// Descriptors and query embeddings enter the similarity stage (App. D.2
// step 3) as unit vectors, so a dot product is the cosine.  For the
// FP32-accurate tensor-core path every unit row x is also stored as
//   x_hi = FP16(x)  (11 significant bits),  x_lo = FP16(2^11 (x - x_hi)),
// so that x_hi*y_hi + 2^-11 (x_hi*y_lo + x_lo*y_hi) reproduces x*y to about
// 2^-22 relative per product (the dropped x_lo*y_lo term and the rounding of
// x_lo are both of that order).  x - x_hi is exact in FP32 and the power-of-two
// scale is exact; it lifts the residual out of FP16's subnormal range.  Unit
// rows have |x| <= 1, far inside FP16's range.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include "farm_internal.h"

namespace farm {
namespace {

__device__ __forceinline__ uint16_t half_bits(__half h) { return *reinterpret_cast<uint16_t *>(&h); }

// One warp per row: the sum of squares from float4 loads (four in flight per
// lane), then the unit row written to each requested copy.  split >= 0: a
// destination row below split gets the FP32 and BF16 copies only, one at or
// above it the FP16 split only (a batch whose last rows run the FP32-accurate
// similarity); split < 0: every requested copy of every row.
__global__ void normalize_rows_kernel(const float *__restrict__ src, const int32_t *__restrict__ dst_rows,
                                      int64_t rows, int32_t dim, int32_t dim_pad,
                                      float *__restrict__ dst32, uint16_t *__restrict__ dst_hi,
                                      uint16_t *__restrict__ dst_lo, uint16_t *__restrict__ dst_bf16,
                                      int64_t split, int32_t *err, int err_bit)
{
    const int lane = threadIdx.x & 31;
    const int64_t row = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (row >= rows) return;
    const float *x = src + row * (int64_t)dim;
    // float4 loads and stores where every row starts on a 16-byte boundary
    // (8 bytes for the 16-bit copies)
    auto al = [](const void *q, uintptr_t a) { return q == nullptr || (reinterpret_cast<uintptr_t>(q) & (a - 1)) == 0; };
    const bool vec = ((dim | dim_pad) & 3) == 0 && al(src, 16) && al(dst32, 16) && al(dst_hi, 8) && al(dst_lo, 8) &&
                     al(dst_bf16, 8);
    float ss = 0.f;
    if (vec) {
        const float4 *x4 = reinterpret_cast<const float4 *>(x);
        const int n4 = dim >> 2;
        float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
        for (int k = lane; k < n4; k += 4 * 32) {
            float4 v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u)
                v[u] = k + u * 32 < n4 ? __ldg(x4 + k + u * 32) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                s0 = fmaf(v[u].x, v[u].x, s0);
                s1 = fmaf(v[u].y, v[u].y, s1);
                s2 = fmaf(v[u].z, v[u].z, s2);
                s3 = fmaf(v[u].w, v[u].w, s3);
            }
        }
        ss = (s0 + s1) + (s2 + s3);
    } else {
        for (int k = lane; k < dim; k += 32) ss = fmaf(x[k], x[k], ss);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
    const float nrm = sqrtf(ss);
    const bool bad = !(nrm > 0.f) || !isfinite(nrm);
    if (bad && lane == 0) atomicOr(err, err_bit);
    const int64_t drow = dst_rows ? (int64_t)dst_rows[row] : row;
    const int64_t base = drow * (int64_t)dim_pad;
    if (split >= 0) {
        if (drow >= split) dst32 = nullptr, dst_bf16 = nullptr;
        else dst_hi = nullptr;
    }
    if (vec) {
        // dim_pad is a multiple of 4: groups of four entries, zero past dim
        const int n4 = dim_pad >> 2;
        const float4 *x4 = reinterpret_cast<const float4 *>(x);
        for (int k = lane; k < n4; k += 32) {
            float4 a = make_float4(0.f, 0.f, 0.f, 0.f);
            if (4 * k < dim && !bad) {
                a = __ldg(x4 + k);
                a.x = a.x / nrm; a.y = a.y / nrm; a.z = a.z / nrm; a.w = a.w / nrm;
            }
            if (dst32) reinterpret_cast<float4 *>(dst32 + base)[k] = a;
            const float v[4] = {a.x, a.y, a.z, a.w};
            if (dst_hi) {
                uint16_t h[4], l[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const __half hi = __float2half_rn(v[u]);
                    h[u] = half_bits(hi);
                    l[u] = half_bits(__float2half_rn((v[u] - __half2float(hi)) * 2048.f));
                }
                reinterpret_cast<uint2 *>(dst_hi + base)[k] =
                    make_uint2((uint32_t)h[0] | (uint32_t)h[1] << 16, (uint32_t)h[2] | (uint32_t)h[3] << 16);
                reinterpret_cast<uint2 *>(dst_lo + base)[k] =
                    make_uint2((uint32_t)l[0] | (uint32_t)l[1] << 16, (uint32_t)l[2] | (uint32_t)l[3] << 16);
            }
            if (dst_bf16) {
                uint16_t b[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const __nv_bfloat16 t = __float2bfloat16_rn(v[u]);
                    b[u] = *reinterpret_cast<const uint16_t *>(&t);
                }
                reinterpret_cast<uint2 *>(dst_bf16 + base)[k] =
                    make_uint2((uint32_t)b[0] | (uint32_t)b[1] << 16, (uint32_t)b[2] | (uint32_t)b[3] << 16);
            }
        }
        return;
    }
    for (int k = lane; k < dim_pad; k += 32) {
        float v = (k < dim && !bad) ? x[k] / nrm : 0.f;
        if (dst32) dst32[base + k] = v;
        if (dst_hi) {
            const __half hi = __float2half_rn(v);
            dst_hi[base + k] = half_bits(hi);
            dst_lo[base + k] = half_bits(__float2half_rn((v - __half2float(hi)) * 2048.f));
        }
        if (dst_bf16) {
            __nv_bfloat16 b = __float2bfloat16_rn(v);
            dst_bf16[base + k] = *reinterpret_cast<uint16_t *>(&b);
        }
    }
}

// One thread per (object, view).
__global__ void prepare_views_kernel(const float *__restrict__ v, const float *__restrict__ pos, int64_t n,
                                     int32_t n_views, float *__restrict__ out)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n * n_views) return;
    const int64_t j = t / n_views;
    const int32_t w = (int32_t)(t - j * n_views);
    const int64_t plane = (int64_t)n_views * n;
    const int64_t at = (int64_t)w * n + j;
    float ox = v[0 * plane + at], oy = v[1 * plane + at], oz = v[2 * plane + at];
    float fx = v[3 * plane + at], fy = v[4 * plane + at], fz = v[5 * plane + at];
    float fn = sqrtf(fx * fx + fy * fy + fz * fz);
    float rx = 0.f, ry = 0.f;
    if (fn > 0.f && isfinite(fn)) {
        fx /= fn; fy /= fn; fz /= fn;
        rx = fy; ry = -fx;
        float rn = sqrtf(rx * rx + ry * ry);
        if (rn > 0.f) {
            rx /= rn; ry /= rn;
        } else {
            fx = fy = fz = 0.f; rx = ry = 0.f;
        }
    } else {
        fx = fy = fz = 0.f;
    }
    // the object's own depth and image coordinate in this view, which every
    // relation of the object against a landmark in this view compares with
    const float dex = pos[j] - ox, dey = pos[n + j] - oy, dez = pos[2 * n + j] - oz;
    const float ze = dex * fx + dey * fy + dez * fz;
    const float ue = (dex * rx + dey * ry) / ze;
    float *o = out + t * kViewStride;
    o[0] = ox; o[1] = oy; o[2] = oz;
    o[3] = fx; o[4] = fy; o[5] = fz;
    o[6] = rx; o[7] = ry;
    o[8] = ze; o[9] = ue; o[10] = 0.f; o[11] = 0.f;
}

// One warp per unit row: scale = max|x| / 448 (the largest finite E4M3
// value), q = E4M3(x / scale) with saturation.
__global__ void quantize_fp8_rows_kernel(const float *__restrict__ src, int64_t rows, int32_t dim_pad,
                                         uint8_t *__restrict__ dst, float *__restrict__ scale)
{
    const int lane = threadIdx.x & 31;
    const int64_t row = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (row >= rows) return;
    const float *x = src + row * (int64_t)dim_pad;
    float amax = 0.f;
    for (int k = lane; k < dim_pad; k += 32) amax = fmaxf(amax, fabsf(x[k]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
    const float sc = amax > 0.f ? amax / 448.f : 1.f;
    if (lane == 0) scale[row] = sc;
    uint8_t *d = dst + row * (int64_t)dim_pad;
    for (int k = lane; k < dim_pad; k += 32) {
        const __nv_fp8_e4m3 v(x[k] / sc);
        d[k] = v.__x;
    }
}

}  // namespace

cudaError_t launch_quantize_fp8_rows(const float *src, int64_t rows, int32_t dim_pad, uint8_t *dst, float *scale,
                                     cudaStream_t s)
{
    if (rows <= 0) return cudaSuccess;
    const int warps = 8;
    quantize_fp8_rows_kernel<<<(unsigned)((rows + warps - 1) / warps), warps * 32, 0, s>>>(src, rows, dim_pad, dst,
                                                                                             scale);
    return cudaGetLastError();
}

cudaError_t launch_normalize_rows(const float *src, const int32_t *dst_rows, int64_t rows,
                                  int32_t dim, int32_t dim_pad, float *dst32, uint16_t *dst_hi,
                                  uint16_t *dst_lo, uint16_t *dst_bf16, int32_t *err, int err_bit,
                                  cudaStream_t s, int64_t split)
{
    if (rows <= 0) return cudaSuccess;
    const int warps = 8;
    const int64_t blocks = (rows + warps - 1) / warps;
    normalize_rows_kernel<<<(unsigned)blocks, warps * 32, 0, s>>>(src, dst_rows, rows, dim, dim_pad,
                                                                   dst32, dst_hi, dst_lo, dst_bf16,
                                                                   split, err, err_bit);
    return cudaGetLastError();
}

cudaError_t launch_prepare_views(const float *views_soa, const float *pos, int64_t n, int32_t n_views, float *out,
                                 cudaStream_t s)
{
    const int64_t total = n * n_views;
    if (total <= 0) return cudaSuccess;
    const int th = 256;
    prepare_views_kernel<<<(unsigned)((total + th - 1) / th), th, 0, s>>>(views_soa, pos, n, n_views, out);
    return cudaGetLastError();
}

// Loads the normalisation kernel (modules and functions load lazily on first use).
cudaError_t preload_prep()
{
    cudaFuncAttributes a;
    return cudaFuncGetAttributes(&a, normalize_rows_kernel);
}

}  // namespace farm
