// k_select.cu -- per-row rank selection (App. D.2 step 3 ranks, step 4
// landmark candidates).
//
// For each similarity row the kernel returns the R largest entries in rank
// order: value descending, lower object index first among equal values, i.e.
// exactly the objects of rank 1..R of the definition
//   rank(j) = 1 + #{j' : c_j' > c_j, or c_j' = c_j and j' < j}.
// Target rows keep R = r_tgt candidates (the rank bound of farm_query_batch),
// landmark rows keep R = K_a.
//
// One CTA per row.  Values map to order-preserving 32-bit keys; radix passes
// find the key T of the R-th largest entry and how many entries equal to T
// still belong in the list; one pass appends every key > T (and the entries
// equal to T when all of them belong); otherwise an ordered pass takes the
// first entries equal to T in index order; a bitonic sort over (key, index)
// in shared memory puts the list in rank order.
//
// Rows of up to kRowSmemMax entries are staged once in shared memory (two
// CTAs per SM) and take three passes with 11/11/10-bit digits over shared
// memory; longer rows stay in global memory (four 8-bit passes, L2-resident).
#include "select_common.cuh"

namespace farm {
namespace {

using namespace sel;

constexpr int TH = 512;
constexpr int SORT_MAX = kMaxTargetCands;   // >= kMaxAnchorCands
constexpr int kRowSmemMax = kSelectRowMax;  // entries staged in shared memory (96 KB)

__global__ void __launch_bounds__(TH)
select_rows_global_kernel(const float *__restrict__ S, int64_t ld_s, int32_t n, int64_t n_tgt_rows,
                          int32_t r_tgt, int32_t k_lm, int32_t *__restrict__ tsel_idx,
                          float *__restrict__ tsel_cos, int64_t tsel_row0, int32_t stride_t,
                          int32_t *__restrict__ lsel_idx, float *__restrict__ lsel_cos, int64_t lsel_row0,
                          int32_t stride_l)
{
    __shared__ uint32_t hist[256];
    __shared__ uint64_t cand[SORT_MAX];
    __shared__ int s_misc[TH / 32 + 3];
    const int64_t r = blockIdx.x;
    const float *row = S + r * ld_s;
    if (r < n_tgt_rows) {
        const int64_t o = (tsel_row0 + r) * (int64_t)stride_t;
        select_row_global<TH>(row, n, r_tgt, cand, hist, s_misc, tsel_idx + o, tsel_cos ? tsel_cos + o : nullptr,
                              stride_t, 0.f);
    } else {
        const int64_t o = (lsel_row0 + (r - n_tgt_rows)) * (int64_t)stride_l;
        select_row_global<TH>(row, n, k_lm, cand, hist, s_misc, lsel_idx + o, lsel_cos ? lsel_cos + o : nullptr,
                              stride_l, 0.f);
    }
}


// Bitonic sort of P (a power of two <= TH) 64-bit keys in shared memory,
// descending, one element per thread.  Stages whose partners lie in the same
// warp synchronise the warp only.
__device__ __forceinline__ void bitonic_desc_warp(uint64_t *cand, int P)
{
    const int i = threadIdx.x;
    int prev_j = TH;
    for (int k = 2; k <= P; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            if (j >= 32 || prev_j >= 32) __syncthreads();
            else __syncwarp();
            if (i < P) {
                const int ixj = i ^ j;
                if (ixj > i) {
                    const uint64_t a = cand[i], b = cand[ixj];
                    const bool desc = (i & k) == 0;
                    if (desc ? (a < b) : (a > b)) { cand[i] = b; cand[ixj] = a; }
                }
            }
            prev_j = j;
        }
    }
    __syncthreads();
}

constexpr int kVecHalf = kRowSmemMax / 8 / TH;   // float4 loads per thread per batch (two batches)

// The R largest entries of one row (n <= kRowSmemMax, `row` 16-byte
// aligned) staged in shared memory (`keys`, dynamic), written in rank order
// to oi / oc (nullable) [0, out_stride) as write_list maps positions.  Among
// equal values the lower position comes first, so a row whose position order
// agrees with object-index order among equal values (a row of S, or chunk
// lists laid end to end) yields the rank order of the definition.
__device__ __forceinline__ void select_row_smem(const float *__restrict__ row, int n, int R, int32_t idx_base,
                                                const int32_t *__restrict__ idx_map, int32_t *__restrict__ oi,
                                                float *__restrict__ oc, int out_stride, float pad)
{
    extern __shared__ uint32_t keys[];
    __shared__ uint32_t hist[2048];
    __shared__ uint64_t cand[SORT_MAX];
    __shared__ uint32_t wsum[TH / 32];
    __shared__ uint32_t s_bin, s_rem, s_cnt;
    __shared__ int s_app, s_warp[TH / 32];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int n4 = n & ~3;

    // issue the row's loads in two batches of kVecHalf float4 per thread, then
    // histogram the top 11 bits of each key
    for (int i = tid; i < 2048; i += TH) hist[i] = 0;
    __syncthreads();
#pragma unroll
    for (int half = 0; half < 2; ++half) {
        float4 buf[kVecHalf];
#pragma unroll
        for (int u = 0; u < kVecHalf; ++u) {
            const int i = ((half * kVecHalf + u) * TH + tid) * 4;
            buf[u] = i < n4 ? __ldg(reinterpret_cast<const float4 *>(row + i)) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int u = 0; u < kVecHalf; ++u) {
            const int i = ((half * kVecHalf + u) * TH + tid) * 4;
            if (i < n4) {
                const uint4 k = make_uint4(order_key(buf[u].x), order_key(buf[u].y), order_key(buf[u].z),
                                           order_key(buf[u].w));
                *reinterpret_cast<uint4 *>(keys + i) = k;
                atomicAdd(&hist[k.x >> 21], 1u);
                atomicAdd(&hist[k.y >> 21], 1u);
                atomicAdd(&hist[k.z >> 21], 1u);
                atomicAdd(&hist[k.w >> 21], 1u);
            }
        }
    }
    if (tid < n - n4) {
        const uint32_t k = order_key(row[n4 + tid]);
        keys[n4 + tid] = k;
        atomicAdd(&hist[k >> 21], 1u);
    }
    __syncthreads();
    find_bucket<2048, TH>(hist, (uint32_t)R, wsum, &s_bin, &s_rem, &s_cnt);
    const uint32_t b1 = s_bin;
    uint32_t remaining = s_rem;
    const int nv = (n + 3) >> 2;   // uint4 groups (the tail group is masked by index)
    // second digit: bits 10..20 among keys whose top digit is b1
    for (int i = tid; i < 2048; i += TH) hist[i] = 0;
    __syncthreads();
    for (int g = tid; g < nv; g += TH) {
        const uint4 k = reinterpret_cast<const uint4 *>(keys)[g];
        const uint32_t kk[4] = {k.x, k.y, k.z, k.w};
#pragma unroll
        for (int c = 0; c < 4; ++c)
            if (4 * g + c < n && (kk[c] >> 21) == b1) atomicAdd(&hist[(kk[c] >> 10) & 2047u], 1u);
    }
    __syncthreads();
    find_bucket<2048, TH>(hist, remaining, wsum, &s_bin, &s_rem, &s_cnt);
    const uint32_t p2 = (b1 << 11) | s_bin;     // top 22 bits
    remaining = s_rem;
    // third digit: bits 0..9
    for (int i = tid; i < 1024; i += TH) hist[i] = 0;
    __syncthreads();
    for (int g = tid; g < nv; g += TH) {
        const uint4 k = reinterpret_cast<const uint4 *>(keys)[g];
        const uint32_t kk[4] = {k.x, k.y, k.z, k.w};
#pragma unroll
        for (int c = 0; c < 4; ++c)
            if (4 * g + c < n && (kk[c] >> 10) == p2) atomicAdd(&hist[kk[c] & 1023u], 1u);
    }
    __syncthreads();
    find_bucket<1024, TH>(hist, remaining, wsum, &s_bin, &s_rem, &s_cnt);
    const uint32_t T = (p2 << 10) | s_bin;
    remaining = s_rem;
    const bool take_all_eq = s_cnt == remaining;
    const int n_gt = R - (int)remaining;

    if (tid == 0) s_app = 0;
    __syncthreads();
    for (int g = tid; g < nv; g += TH) {
        const uint4 k = reinterpret_cast<const uint4 *>(keys)[g];
        const uint32_t kk[4] = {k.x, k.y, k.z, k.w};
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int i = 4 * g + c;
            if (i < n && (kk[c] > T || (take_all_eq && kk[c] == T))) {
                const int pos = atomicAdd(&s_app, 1);
                cand[pos] = cand_word(kk[c], i);
            }
        }
    }
    __syncthreads();
    if (!take_all_eq) {
        int taken = 0;
        for (int base = 0; base < n && taken < (int)remaining; base += TH) {
            const int j = base + tid;
            const bool eq = j < n && keys[j] == T;
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
                if (pos < (int)remaining)
                    cand[n_gt + pos] = cand_word(T, j);
            }
            taken += tot;
            __syncthreads();
        }
    }
    int P = 1;
    while (P < R) P <<= 1;
    for (int i = R + tid; i < P; i += TH) cand[i] = 0ull;
    bitonic_desc_warp(cand, P);
    write_list<TH>(cand, R, idx_base, idx_map, oi, oc, out_stride, pad);
    __syncthreads();   // the shared arrays are reused by the block's next call
}

__global__ void __launch_bounds__(TH, 2)
select_rows_smem_kernel(const float *__restrict__ S, int64_t ld_s, int32_t n, int64_t n_tgt_rows,
                        int32_t r_tgt, int32_t k_lm, int32_t *__restrict__ tsel_idx,
                        float *__restrict__ tsel_cos, int64_t tsel_row0, int32_t stride_t,
                        int32_t *__restrict__ lsel_idx, float *__restrict__ lsel_cos, int64_t lsel_row0,
                        int32_t stride_l)
{
    const int64_t r = blockIdx.x;
    const bool is_tgt = r < n_tgt_rows;
    if (is_tgt) {
        select_row_smem(S + r * ld_s, n, r_tgt, 0, nullptr, tsel_idx + (tsel_row0 + r) * (int64_t)stride_t,
                        tsel_cos ? tsel_cos + (tsel_row0 + r) * (int64_t)stride_t : nullptr, stride_t, 0.f);
    } else {
        const int64_t l = lsel_row0 + (r - n_tgt_rows);
        select_row_smem(S + r * ld_s, n, k_lm, 0, nullptr, lsel_idx + l * (int64_t)stride_l,
                        lsel_cos ? lsel_cos + l * (int64_t)stride_l : nullptr, stride_l, 0.f);
    }
}

// Grouped select: block -> (piece, row, chunk) through the piece table.
__global__ void __launch_bounds__(TH, 2)
select_grouped_kernel(const float *__restrict__ S, const Piece *__restrict__ pieces, int32_t n_pieces,
                      int32_t *__restrict__ tsel_idx, float *__restrict__ tsel_cos, int32_t stride_t,
                      int32_t *__restrict__ lsel_idx, float *__restrict__ lsel_cos, int32_t stride_l,
                      int32_t *__restrict__ tmp_idx, float *__restrict__ tmp_val, int32_t tmp_stride)
{
    const int64_t b = blockIdx.x;
    const Piece pc = pieces[find_piece(pieces, n_pieces, b, [](const Piece &x) { return x.block_begin; })];
    const int64_t local = b - pc.block_begin;
    const int i = (int)(local / pc.chunks), c = (int)(local % pc.chunks);
    const bool is_tgt = i < pc.ntr;
    const int R = is_tgt ? pc.keep_t : pc.keep_l;
    const float *row = S + pc.s_off + (int64_t)i * pc.ld;
    if (pc.chunks == 1) {
        if (is_tgt) {
            const int64_t o = (pc.t_row0 + i) * (int64_t)stride_t;
            select_row_smem(row, pc.n, R, 0, nullptr, tsel_idx + o, tsel_cos ? tsel_cos + o : nullptr, stride_t, 0.f);
        } else {
            const int64_t o = (pc.l_row0 + (i - pc.ntr)) * (int64_t)stride_l;
            select_row_smem(row, pc.n, R, 0, nullptr, lsel_idx + o, lsel_cos ? lsel_cos + o : nullptr, stride_l, 0.f);
        }
    } else {
        const int c0 = c * pc.chunk_len;
        const int len = min(pc.chunk_len, pc.n - c0);
        const int64_t o = pc.tmp_off + ((int64_t)i * pc.chunks + c) * tmp_stride;
        select_row_smem(row + c0, len, min(R, len), c0, nullptr, tmp_idx + o, tmp_val + o, tmp_stride,
                        -__int_as_float(0x7f800000));
    }
}

// Merge of a chunked row: its chunk lists, laid end to end in chunk order,
// list equal values in object-index order, so a select over them with
// position -> index through tmp_idx gives the row's rank order.
__global__ void __launch_bounds__(TH, 2)
merge_chunks_kernel(const Piece *__restrict__ pieces, int32_t n_pieces, const int32_t *__restrict__ tmp_idx,
                    const float *__restrict__ tmp_val, int32_t tmp_stride, int32_t *__restrict__ tsel_idx,
                    float *__restrict__ tsel_cos, int32_t stride_t, int32_t *__restrict__ lsel_idx,
                    float *__restrict__ lsel_cos, int32_t stride_l)
{
    const int64_t r = blockIdx.x;
    const Piece pc = pieces[find_piece(pieces, n_pieces, r, [](const Piece &x) { return x.row_begin; })];
    const int i = (int)(r - pc.row_begin);
    if (pc.chunks <= 1 || i >= pc.th0) return;   // unchunked rows, rows of the per-piece or thresholded select
    const int M = pc.chunks * tmp_stride;
    const int64_t o = pc.tmp_off + (int64_t)i * M;
    if (i < pc.ntr) {
        const int64_t w = (pc.t_row0 + i) * (int64_t)stride_t;
        select_row_smem(tmp_val + o, M, pc.keep_t, 0, tmp_idx + o, tsel_idx + w, tsel_cos ? tsel_cos + w : nullptr,
                        stride_t, 0.f);
    } else {
        const int64_t w = (pc.l_row0 + (i - pc.ntr)) * (int64_t)stride_l;
        select_row_smem(tmp_val + o, M, pc.keep_l, 0, tmp_idx + o, lsel_idx + w, lsel_cos ? lsel_cos + w : nullptr,
                        stride_l, 0.f);
    }
}

cudaError_t set_smem(const void *fn, int32_t smem_n, size_t *bytes)
{
    *bytes = (size_t)((smem_n + 3) & ~3) * sizeof(uint32_t);
    return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)*bytes);
}

}  // namespace

cudaError_t launch_select_rows_ex(const float *S, int64_t ld_s, int64_t n, int64_t rows, int64_t n_tgt_rows,
                                  int32_t r_tgt, int32_t k_lm, int32_t *tsel_idx, float *tsel_cos, int64_t tsel_row0,
                                  int32_t stride_t, int32_t *lsel_idx, float *lsel_cos, int64_t lsel_row0,
                                  int32_t stride_l, cudaStream_t s)
{
    if (rows <= 0) return cudaSuccess;
    if (r_tgt < 1 || r_tgt > SORT_MAX || r_tgt > n || k_lm < 1 || k_lm > kMaxAnchorCands ||
        k_lm > n || n > 0x7fffffff)
        return cudaErrorInvalidValue;
    if (n <= kRowSmemMax && (ld_s % 4) == 0 && ((uintptr_t)S & 15u) == 0) {
        const size_t smem = (size_t)((n + 3) & ~3) * sizeof(uint32_t);
        cudaError_t e = cudaFuncSetAttribute(select_rows_smem_kernel,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        select_rows_smem_kernel<<<(unsigned)rows, TH, smem, s>>>(S, ld_s, (int32_t)n, n_tgt_rows, r_tgt, k_lm,
                                                                  tsel_idx, tsel_cos, tsel_row0, stride_t,
                                                                  lsel_idx, lsel_cos, lsel_row0, stride_l);
    } else {
        select_rows_global_kernel<<<(unsigned)rows, TH, 0, s>>>(S, ld_s, (int32_t)n, n_tgt_rows, r_tgt, k_lm,
                                                                 tsel_idx, tsel_cos, tsel_row0, stride_t,
                                                                 lsel_idx, lsel_cos, lsel_row0, stride_l);
    }
    return cudaGetLastError();
}

cudaError_t launch_select_rows(const float *S, int64_t ld_s, int64_t n, int64_t rows,
                               int64_t n_tgt_rows, int32_t r_tgt, int32_t k_lm,
                               int32_t *tsel_idx, float *tsel_cos, int64_t tsel_row0,
                               int32_t stride_t, int32_t *lsel_idx, int64_t lsel_row0,
                               int32_t stride_l, cudaStream_t s)
{
    return launch_select_rows_ex(S, ld_s, n, rows, n_tgt_rows, r_tgt, k_lm, tsel_idx, tsel_cos, tsel_row0, stride_t,
                                 lsel_idx, nullptr, lsel_row0, stride_l, s);
}

cudaError_t launch_select_grouped(const float *S, const Piece *pieces, int32_t n_pieces, int64_t total_blocks,
                                  int32_t smem_n, int32_t *tsel_idx, float *tsel_cos, int32_t stride_t,
                                  int32_t *lsel_idx, float *lsel_cos, int32_t stride_l, int32_t *tmp_idx,
                                  float *tmp_val, int32_t tmp_stride, cudaStream_t s)
{
    if (total_blocks <= 0) return cudaSuccess;
    if (n_pieces < 1 || smem_n < 1 || smem_n > kRowSmemMax || total_blocks > 0x7fffffff || (tmp_stride & 3) != 0 ||
        ((uintptr_t)S & 15u) != 0)
        return cudaErrorInvalidValue;
    size_t smem = 0;
    cudaError_t e = set_smem((const void *)select_grouped_kernel, smem_n, &smem);
    if (e != cudaSuccess) return e;
    select_grouped_kernel<<<(unsigned)total_blocks, TH, smem, s>>>(S, pieces, n_pieces, tsel_idx, tsel_cos,
                                                                   stride_t, lsel_idx, lsel_cos, stride_l, tmp_idx,
                                                                   tmp_val, tmp_stride);
    return cudaGetLastError();
}

cudaError_t launch_merge_chunks(const Piece *pieces, int32_t n_pieces, int64_t total_rows, int32_t smem_n,
                                const int32_t *tmp_idx, const float *tmp_val, int32_t tmp_stride,
                                int32_t *tsel_idx, float *tsel_cos, int32_t stride_t, int32_t *lsel_idx,
                                float *lsel_cos, int32_t stride_l, cudaStream_t s)
{
    if (total_rows <= 0) return cudaSuccess;
    if (n_pieces < 1 || smem_n < 1 || smem_n > kRowSmemMax || total_rows > 0x7fffffff || (tmp_stride & 3) != 0)
        return cudaErrorInvalidValue;
    size_t smem = 0;
    cudaError_t e = set_smem((const void *)merge_chunks_kernel, smem_n, &smem);
    if (e != cudaSuccess) return e;
    merge_chunks_kernel<<<(unsigned)total_rows, TH, smem, s>>>(pieces, n_pieces, tmp_idx, tmp_val, tmp_stride,
                                                               tsel_idx, tsel_cos, stride_t, lsel_idx, lsel_cos,
                                                               stride_l);
    return cudaGetLastError();
}

// Loads the per-row select kernels (modules and functions load lazily on first use).
cudaError_t preload_select_rows()
{
    cudaFuncAttributes a;
    cudaError_t e = cudaFuncGetAttributes(&a, select_rows_smem_kernel);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, select_rows_global_kernel);
    return e;
}

}  // namespace farm
