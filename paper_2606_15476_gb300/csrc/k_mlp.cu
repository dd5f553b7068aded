// k_mlp.cu -- kernels of the learned descriptor prefilter: a two-layer MLP
//   f(x) = normalize(W2 gelu(W1 x + b1) + b2),   x in R^D, W1: H x D, W2: P x H,
// its forward and backward passes for training on (query row, descriptor,
// oracle cosine) pairs with the loss
//   L = sum_i w_i (f(q_i) . f(d_i) - y_i)^2 / sum_i w_i,
// and an Adam update.  The contractions of training and inference run on the
// tensor cores (BF16 operands, FP32 accumulation) through the similarity
// kernel of k_sim_tc.cu, fed by the gathers, transposes and BF16 conversions
// below; the tiled FP32 GEMM on the CUDA cores here is the FP32 reference
// arithmetic of farm_mlp_loss_grad and farm_mlp_embed.  Elementwise steps
// (bias, GELU in its exact erf form, normalisation, the loss and their
// gradients, Adam) are FP32 on the CUDA cores.
#include <cuda_bf16.h>

#include "farm_internal.h"

namespace farm {
namespace {

// C[M,N] (ldc) = alpha * op(A) op(B) + beta * C.
//   TA = false: A is [M, K] (lda), K contiguous;  TA = true: A is [K, M] (lda), M contiguous.
//   TB = false: B is [N, K] (ldb), K contiguous;  TB = true: B is [K, N] (ldb), N contiguous.
// 64 x 64 tiles, 16-wide K slices, 256 threads with 4 x 4 outputs each; all
// bounds checked (M, N, K arbitrary).
template <bool TA, bool TB>
__global__ void __launch_bounds__(256)
gemm_f32_kernel(int M, int N, int K, float alpha, const float *__restrict__ A, int lda,
                const float *__restrict__ B, int ldb, float beta, float *__restrict__ C, int ldc)
{
    __shared__ float As[16][64 + 1];
    __shared__ float Bs[16][64 + 1];
    const int tid = threadIdx.x;
    const int m0 = blockIdx.y * 64, n0 = blockIdx.x * 64;
    const int tx = tid & 15, ty = tid >> 4;
    float acc[4][4] = {};
    for (int k0 = 0; k0 < K; k0 += 16) {
        // 64 x 16 elements per operand, 4 per thread
        for (int e = tid; e < 64 * 16; e += 256) {
            int mm, kk;
            if (TA) { mm = e & 63; kk = e >> 6; } else { kk = e & 15; mm = e >> 4; }
            const int gm = m0 + mm, gk = k0 + kk;
            float v = 0.f;
            if (gm < M && gk < K) v = TA ? A[(int64_t)gk * lda + gm] : A[(int64_t)gm * lda + gk];
            As[kk][mm] = v;
        }
        for (int e = tid; e < 64 * 16; e += 256) {
            int nn, kk;
            if (TB) { nn = e & 63; kk = e >> 6; } else { kk = e & 15; nn = e >> 4; }
            const int gn = n0 + nn, gk = k0 + kk;
            float v = 0.f;
            if (gn < N && gk < K) v = TB ? B[(int64_t)gk * ldb + gn] : B[(int64_t)gn * ldb + gk];
            Bs[kk][nn] = v;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            float a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx * 4 + j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int gm = m0 + ty * 4 + i;
        if (gm >= M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int gn = n0 + tx * 4 + j;
            if (gn >= N) continue;
            float *c = C + (int64_t)gm * ldc + gn;
            *c = alpha * acc[i][j] + (beta != 0.f ? beta * *c : 0.f);
        }
    }
}

__device__ __forceinline__ float gelu(float x) { return 0.5f * x * (1.f + erff(x * 0.70710678118654752f)); }

__device__ __forceinline__ float gelu_grad(float x)
{
    const float cdf = 0.5f * (1.f + erff(x * 0.70710678118654752f));
    const float pdf = 0.39894228040143268f * expf(-0.5f * x * x);
    return cdf + x * pdf;
}

__device__ __forceinline__ uint16_t bf16_bits(float x)
{
    __nv_bfloat16 b = __float2bfloat16_rn(x);
    return *reinterpret_cast<uint16_t *>(&b);
}

// h[r, j] += b[j] (pre-activation kept), a[r, j] = gelu(h[r, j]) (and its BF16 copy ab, nullable).
__global__ void bias_gelu_kernel(float *__restrict__ h, const float *__restrict__ b, float *__restrict__ a,
                                 uint16_t *__restrict__ ab, int64_t rows, int cols)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= rows * cols) return;
    const float v = h[i] + b[i % cols];
    h[i] = v;
    const float g = gelu(v);
    a[i] = g;
    if (ab) ab[i] = bf16_bits(g);
}

// z[r, :] += b, then e = z / |z| (norm kept); one warp per row.
__global__ void bias_normalize_kernel(float *__restrict__ z, const float *__restrict__ b, float *__restrict__ e,
                                      float *__restrict__ norm, int64_t rows, int cols)
{
    const int lane = threadIdx.x & 31;
    const int64_t r = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (r >= rows) return;
    float *zr = z + r * cols;
    float ss = 0.f;
    for (int j = lane; j < cols; j += 32) {
        const float v = zr[j] + b[j];
        zr[j] = v;
        ss = fmaf(v, v, ss);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
    const float nrm = fmaxf(sqrtf(ss), 1e-20f);
    if (lane == 0 && norm) norm[r] = nrm;
    for (int j = lane; j < cols; j += 32) e[r * cols + j] = zr[j] / nrm;
}

// Per pair: s = eq . ed, loss += w (s - y)^2 / wsum, deq = g ed, ded = g eq
// with g = 2 w (s - y) / wsum.  One warp per pair.
__global__ void pair_loss_kernel(const float *__restrict__ eq, const float *__restrict__ ed,
                                 const float *__restrict__ y, const float *__restrict__ w, float wsum, int64_t pairs,
                                 int cols, float *__restrict__ deq, float *__restrict__ ded, float *__restrict__ loss)
{
    const int lane = threadIdx.x & 31;
    const int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (i >= pairs) return;
    const float *a = eq + i * cols, *b = ed + i * cols;
    float s = 0.f;
    for (int j = lane; j < cols; j += 32) s = fmaf(a[j], b[j], s);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    const float wi = w ? w[i] : 1.f;
    const float r = s - y[i];
    const float g = 2.f * wi * r / wsum;
    if (lane == 0) atomicAdd(loss, wi * r * r / wsum);
    for (int j = lane; j < cols; j += 32) {
        deq[i * cols + j] = g * b[j];
        ded[i * cols + j] = g * a[j];
    }
}

// dz = (de - e (e . de)) / |z|; one warp per row (in place on de).
__global__ void normalize_backward_kernel(const float *__restrict__ e, const float *__restrict__ norm,
                                          float *__restrict__ de, int64_t rows, int cols)
{
    const int lane = threadIdx.x & 31;
    const int64_t r = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (r >= rows) return;
    const float *er = e + r * cols;
    float *dr = de + r * cols;
    float dot = 0.f;
    for (int j = lane; j < cols; j += 32) dot = fmaf(er[j], dr[j], dot);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) dot += __shfl_xor_sync(0xffffffffu, dot, o);
    const float inv = 1.f / norm[r];
    for (int j = lane; j < cols; j += 32) dr[j] = (dr[j] - er[j] * dot) * inv;
}

// da *= gelu'(h) in place.
__global__ void gelu_backward_kernel(const float *__restrict__ h, float *__restrict__ da, int64_t count)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) da[i] *= gelu_grad(h[i]);
}

// out[j] += sum_r x[r, j]: block (32 columns x 8 row lanes) over a chunk of
// 256 rows, shared-memory reduction, one atomic per column and block.
__global__ void colsum_kernel(const float *__restrict__ x, int64_t rows, int cols, float *__restrict__ out)
{
    __shared__ float part[8][33];
    const int c = blockIdx.x * 32 + (threadIdx.x & 31);
    const int lane_r = threadIdx.x >> 5;
    const int64_t r0 = (int64_t)blockIdx.y * 256;
    float s = 0.f;
    if (c < cols)
        for (int64_t r = r0 + lane_r; r < min(rows, r0 + 256); r += 8) s += x[r * cols + c];
    part[lane_r][threadIdx.x & 31] = s;
    __syncthreads();
    if (lane_r == 0 && c < cols) {
        float t = 0.f;
        for (int i = 0; i < 8; ++i) t += part[i][threadIdx.x & 31];
        atomicAdd(out + c, t);
    }
}

__global__ void to_bf16_kernel(const float *__restrict__ x, int64_t count, uint16_t *__restrict__ y)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    __nv_bfloat16 b = __float2bfloat16_rn(x[i]);
    y[i] = *reinterpret_cast<uint16_t *>(&b);
}

// dst[r, :] = src[idx[r], :] (rows of `cols` floats, source leading dimension lds).
__global__ void gather_rows_kernel(const float *__restrict__ src, int lds, const int32_t *__restrict__ idx,
                                   int64_t rows, int cols, float *__restrict__ dst)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= rows * cols) return;
    const int64_t r = i / cols;
    const int c = (int)(i - r * cols);
    dst[i] = src[(int64_t)idx[r] * lds + c];
}

// dst[r, 0:cols] = src_r[0:cols] with src_r = base[sel[r]] + idx[r] * lds (BF16 rows;
// sel null: table entry 0), 16 bytes per thread (cols and the strides multiples of 8).
__global__ void gather_rows_bf16_kernel(const uint16_t *const *__restrict__ base, const int32_t *__restrict__ sel,
                                        const int32_t *__restrict__ idx, int64_t lds, int64_t rows, int cols,
                                        uint16_t *__restrict__ dst, int64_t ldd)
{
    const int per_row = cols >> 3;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= rows * per_row) return;
    const int64_t r = i / per_row;
    const int c = (int)(i - r * per_row);
    const uint16_t *src = base[sel ? sel[r] : 0] + (int64_t)idx[r] * lds;
    reinterpret_cast<uint4 *>(dst + r * ldd)[c] = reinterpret_cast<const uint4 *>(src)[c];
}

// dst[c, col0 + r] = bf16(src[r, c]) for r < rows, c < cols (32 x 32 tiles
// through shared memory: reads along rows of src, writes along rows of dst).
template <class T>
__global__ void transpose_bf16_kernel(const T *__restrict__ src, int64_t lds, int64_t rows, int cols,
                                      uint16_t *__restrict__ dst, int64_t ldd, int64_t col0)
{
    __shared__ uint16_t tile[32][33];
    const int64_t r0 = (int64_t)blockIdx.y * 32;
    const int c0 = blockIdx.x * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;    // 32 x 8 threads
    for (int k = ty; k < 32; k += 8) {
        const int64_t r = r0 + k;
        const int c = c0 + tx;
        uint16_t v = 0;
        if (r < rows && c < cols) {
            if constexpr (sizeof(T) == 4) v = bf16_bits(src[r * lds + c]);
            else v = src[r * lds + c];
        }
        tile[k][tx] = v;
    }
    __syncthreads();
    for (int k = ty; k < 32; k += 8) {
        const int c = c0 + k;
        const int64_t r = r0 + tx;
        if (c < cols && r < rows) dst[(int64_t)c * ldd + col0 + r] = tile[tx][k];
    }
}

// dst[r, c] = bf16(src[r, c]) for c < cols, 0 for cols <= c < ldd.
__global__ void to_bf16_padded_kernel(const float *__restrict__ src, int64_t rows, int cols, uint16_t *__restrict__ dst,
                                      int ldd)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= rows * ldd) return;
    const int64_t r = i / ldd;
    const int c = (int)(i - r * ldd);
    dst[i] = c < cols ? bf16_bits(src[r * cols + c]) : (uint16_t)0;
}

// Adam with bias correction (step t >= 1).
__global__ void adam_kernel(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                            float *__restrict__ v, int64_t count, float lr, float b1, float b2, float eps, int t)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float mh = mi / (1.f - powf(b1, (float)t));
    const float vh = vi / (1.f - powf(b2, (float)t));
    p[i] -= lr * mh / (sqrtf(vh) + eps);
}

unsigned blocks_for(int64_t n, int th) { return (unsigned)((n + th - 1) / th); }

}  // namespace

cudaError_t mlp_gemm(bool ta, bool tb, int M, int N, int K, float alpha, const float *A, int lda, const float *B,
                     int ldb, float beta, float *C, int ldc, cudaStream_t s)
{
    if (M <= 0 || N <= 0) return cudaSuccess;
    dim3 grid((unsigned)((N + 63) / 64), (unsigned)((M + 63) / 64));
    if (!ta && !tb) gemm_f32_kernel<false, false><<<grid, 256, 0, s>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc);
    else if (!ta && tb) gemm_f32_kernel<false, true><<<grid, 256, 0, s>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc);
    else if (ta && !tb) gemm_f32_kernel<true, false><<<grid, 256, 0, s>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc);
    else gemm_f32_kernel<true, true><<<grid, 256, 0, s>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc);
    return cudaGetLastError();
}

cudaError_t mlp_bias_gelu(float *h, const float *b, float *a, int64_t rows, int cols, cudaStream_t s,
                          uint16_t *ab)
{
    if (rows * cols <= 0) return cudaSuccess;
    bias_gelu_kernel<<<blocks_for(rows * cols, 256), 256, 0, s>>>(h, b, a, ab, rows, cols);
    return cudaGetLastError();
}

cudaError_t mlp_gather_rows_bf16(const uint16_t *const *base, const int32_t *sel, const int32_t *idx, int64_t lds,
                                 int64_t rows, int cols, uint16_t *dst, int64_t ldd, cudaStream_t s)
{
    if (rows * cols <= 0) return cudaSuccess;
    if ((cols & 7) || (lds & 7) || (ldd & 7) || (reinterpret_cast<uintptr_t>(dst) & 15)) return cudaErrorInvalidValue;
    gather_rows_bf16_kernel<<<blocks_for(rows * (cols >> 3), 256), 256, 0, s>>>(base, sel, idx, lds, rows, cols, dst,
                                                                                ldd);
    return cudaGetLastError();
}

cudaError_t mlp_transpose_bf16(const float *src32, const uint16_t *src16, int64_t lds, int64_t rows, int cols,
                               uint16_t *dst, int64_t ldd, int64_t col0, cudaStream_t s)
{
    if (rows <= 0 || cols <= 0) return cudaSuccess;
    dim3 grid((unsigned)((cols + 31) / 32), (unsigned)((rows + 31) / 32));
    if (src32) transpose_bf16_kernel<float><<<grid, 256, 0, s>>>(src32, lds, rows, cols, dst, ldd, col0);
    else transpose_bf16_kernel<uint16_t><<<grid, 256, 0, s>>>(src16, lds, rows, cols, dst, ldd, col0);
    return cudaGetLastError();
}

cudaError_t mlp_to_bf16_padded(const float *src, int64_t rows, int cols, uint16_t *dst, int ldd, cudaStream_t s)
{
    if (rows <= 0 || ldd <= 0) return cudaSuccess;
    if (ldd < cols) return cudaErrorInvalidValue;
    to_bf16_padded_kernel<<<blocks_for(rows * ldd, 256), 256, 0, s>>>(src, rows, cols, dst, ldd);
    return cudaGetLastError();
}

cudaError_t mlp_bias_normalize(float *z, const float *b, float *e, float *norm, int64_t rows, int cols,
                               cudaStream_t s)
{
    if (rows <= 0) return cudaSuccess;
    bias_normalize_kernel<<<blocks_for(rows, 8), 256, 0, s>>>(z, b, e, norm, rows, cols);
    return cudaGetLastError();
}

cudaError_t mlp_pair_loss(const float *eq, const float *ed, const float *y, const float *w, float wsum, int64_t pairs,
                          int cols, float *deq, float *ded, float *loss, cudaStream_t s)
{
    if (pairs <= 0) return cudaSuccess;
    pair_loss_kernel<<<blocks_for(pairs, 8), 256, 0, s>>>(eq, ed, y, w, wsum, pairs, cols, deq, ded, loss);
    return cudaGetLastError();
}

cudaError_t mlp_normalize_backward(const float *e, const float *norm, float *de, int64_t rows, int cols,
                                   cudaStream_t s)
{
    if (rows <= 0) return cudaSuccess;
    normalize_backward_kernel<<<blocks_for(rows, 8), 256, 0, s>>>(e, norm, de, rows, cols);
    return cudaGetLastError();
}

cudaError_t mlp_gelu_backward(const float *h, float *da, int64_t count, cudaStream_t s)
{
    if (count <= 0) return cudaSuccess;
    gelu_backward_kernel<<<blocks_for(count, 256), 256, 0, s>>>(h, da, count);
    return cudaGetLastError();
}

cudaError_t mlp_colsum(const float *x, int64_t rows, int cols, float *out, bool accumulate, cudaStream_t s)
{
    if (cols <= 0) return cudaSuccess;
    if (!accumulate) {
        cudaError_t e = cudaMemsetAsync(out, 0, (size_t)cols * sizeof(float), s);
        if (e != cudaSuccess) return e;
    }
    if (rows <= 0) return cudaSuccess;
    dim3 grid((unsigned)((cols + 31) / 32), (unsigned)((rows + 255) / 256));
    colsum_kernel<<<grid, 256, 0, s>>>(x, rows, cols, out);
    return cudaGetLastError();
}

cudaError_t mlp_to_bf16(const float *x, int64_t count, uint16_t *y, cudaStream_t s)
{
    if (count <= 0) return cudaSuccess;
    to_bf16_kernel<<<blocks_for(count, 256), 256, 0, s>>>(x, count, y);
    return cudaGetLastError();
}

cudaError_t mlp_gather_rows(const float *src, int lds, const int32_t *idx, int64_t rows, int cols, float *dst,
                            cudaStream_t s)
{
    if (rows * cols <= 0) return cudaSuccess;
    gather_rows_kernel<<<blocks_for(rows * cols, 256), 256, 0, s>>>(src, lds, idx, rows, cols, dst);
    return cudaGetLastError();
}

cudaError_t mlp_adam(float *p, const float *g, float *m, float *v, int64_t count, float lr, int t, cudaStream_t s)
{
    if (count <= 0) return cudaSuccess;
    adam_kernel<<<blocks_for(count, 256), 256, 0, s>>>(p, g, m, v, count, lr, 0.9f, 0.999f, 1e-8f, t);
    return cudaGetLastError();
}

}  // namespace farm
