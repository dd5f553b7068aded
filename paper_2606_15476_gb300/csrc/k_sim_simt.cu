// k_sim_simt.cu -- descriptor similarity S = Q D^T with FP32 FMA on the CUDA
// cores (App. D.2 step 3: cosine of every query row against every object).
//
// Both operands are row-major with the descriptor dimension contiguous and
// zero-padded to a multiple of kDimAlign.  A CTA of 256 threads computes a
// 128 x 128 tile of S, staging 16-wide K slices of both operands through
// shared memory (double-buffered, transposed so that each thread's 8x8
// register block reads conflict-free).  This path is the plain-FP32 check of
// the tensor-core kernels.
#include "farm_internal.h"

namespace farm {
namespace {

constexpr int BM = 128, BN = 128, BK = 16, TH = 256;

__global__ void __launch_bounds__(TH)
sim_simt_kernel(const float *__restrict__ Q, const float *__restrict__ D, float *__restrict__ S,
                int64_t rows, int64_t n, int32_t ldk, int64_t ld_s)
{
    __shared__ __align__(16) float As[2][BK][BM + 4];
    __shared__ __align__(16) float Bs[2][BK][BN + 4];
    const int tid = threadIdx.x;
    const int64_t m0 = (int64_t)blockIdx.y * BM;
    const int64_t n0 = (int64_t)blockIdx.x * BN;
    // loader mapping: 128 rows x 16 k = 512 float4; 2 per thread per operand
    const int lrow = tid >> 1;            // 0..127
    const int lk = (tid & 1) * 8;         // 0 or 8: two float4 at k = lk, lk+4
    const int64_t arow = m0 + lrow, brow = n0 + lrow;
    const bool aok = arow < rows, bok = brow < n;
    const float *ap = Q + (aok ? arow : 0) * (int64_t)ldk + lk;
    const float *bp = D + (bok ? brow : 0) * (int64_t)ldk + lk;

    const int tx = tid & 15, ty = tid >> 4;   // 16 x 16 threads, 8x8 outputs each
    float acc[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;

    float4 ra0, ra1, rb0, rb1;
    auto gload = [&](int k0) {
        const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
        ra0 = aok ? *reinterpret_cast<const float4 *>(ap + k0) : z;
        ra1 = aok ? *reinterpret_cast<const float4 *>(ap + k0 + 4) : z;
        rb0 = bok ? *reinterpret_cast<const float4 *>(bp + k0) : z;
        rb1 = bok ? *reinterpret_cast<const float4 *>(bp + k0 + 4) : z;
    };
    auto sstore = [&](int buf) {
        As[buf][lk + 0][lrow] = ra0.x; As[buf][lk + 1][lrow] = ra0.y;
        As[buf][lk + 2][lrow] = ra0.z; As[buf][lk + 3][lrow] = ra0.w;
        As[buf][lk + 4][lrow] = ra1.x; As[buf][lk + 5][lrow] = ra1.y;
        As[buf][lk + 6][lrow] = ra1.z; As[buf][lk + 7][lrow] = ra1.w;
        Bs[buf][lk + 0][lrow] = rb0.x; Bs[buf][lk + 1][lrow] = rb0.y;
        Bs[buf][lk + 2][lrow] = rb0.z; Bs[buf][lk + 3][lrow] = rb0.w;
        Bs[buf][lk + 4][lrow] = rb1.x; Bs[buf][lk + 5][lrow] = rb1.y;
        Bs[buf][lk + 6][lrow] = rb1.z; Bs[buf][lk + 7][lrow] = rb1.w;
    };

    const int ktiles = ldk / BK;
    gload(0);
    sstore(0);
    __syncthreads();
    for (int kt = 0; kt < ktiles; ++kt) {
        const int cur = kt & 1;
        if (kt + 1 < ktiles) gload((kt + 1) * BK);
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            float a[8], b[8];
            const float4 a0 = *reinterpret_cast<const float4 *>(&As[cur][kk][ty * 4]);
            const float4 a1 = *reinterpret_cast<const float4 *>(&As[cur][kk][64 + ty * 4]);
            const float4 b0 = *reinterpret_cast<const float4 *>(&Bs[cur][kk][tx * 4]);
            const float4 b1 = *reinterpret_cast<const float4 *>(&Bs[cur][kk][64 + tx * 4]);
            a[0] = a0.x; a[1] = a0.y; a[2] = a0.z; a[3] = a0.w;
            a[4] = a1.x; a[5] = a1.y; a[6] = a1.z; a[7] = a1.w;
            b[0] = b0.x; b[1] = b0.y; b[2] = b0.z; b[3] = b0.w;
            b[4] = b1.x; b[5] = b1.y; b[6] = b1.z; b[7] = b1.w;
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
        if (kt + 1 < ktiles) sstore(cur ^ 1);
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int64_t r = m0 + (i < 4 ? ty * 4 + i : 64 + ty * 4 + (i - 4));
        if (r >= rows) continue;
        float *srow = S + r * ld_s;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int64_t c = n0 + (j < 4 ? tx * 4 + j : 64 + tx * 4 + (j - 4));
            if (c < n) srow[c] = acc[i][j];
        }
    }
}

}  // namespace

cudaError_t launch_sim_simt(const float *q, const float *d, float *S, int64_t rows, int64_t n,
                            int32_t dim_pad, int64_t ld_s, cudaStream_t s)
{
    if (rows <= 0 || n <= 0) return cudaSuccess;
    if (dim_pad % BK != 0) return cudaErrorInvalidValue;
    dim3 grid((unsigned)((n + BN - 1) / BN), (unsigned)((rows + BM - 1) / BM));
    if (grid.y > 65535u) return cudaErrorInvalidConfiguration;
    sim_simt_kernel<<<grid, TH, 0, s>>>(q, d, S, rows, n, dim_pad, ld_s);
    return cudaGetLastError();
}

// Loads the CUDA-core similarity kernel (modules and functions load lazily on first use).
cudaError_t preload_sim_simt()
{
    cudaFuncAttributes a;
    return cudaFuncGetAttributes(&a, sim_simt_kernel);
}

}  // namespace farm
