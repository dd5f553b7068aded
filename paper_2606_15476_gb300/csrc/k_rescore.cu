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
// One CTA per row.  The work is a gather of whole descriptor rows (4.6 KB at
// D = 1152), mostly from L2, so what bounds it is the bytes in flight per SM.
// Rows of up to kTmaDimMax floats: each warp keeps SPW candidate rows in
// flight as bulk asynchronous copies (cp.async.bulk, completion counted on one
// mbarrier per slot) into its own shared-memory slots, and refills a slot as
// soon as its lanes have read it; the dot product is taken from shared memory.
// Longer rows: each warp loads two candidates at a time with four float4 loads
// of each in flight per lane.  The in-band candidates' keys (cosine key, index;
// all distinct) are then ranked: by counting up to 256 of them, else by a
// bitonic sort.
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

constexpr uint32_t WAIT_LIMIT = 1u << 22;   // try_wait polls before giving up (a fraction of a second)
constexpr int kWarps = TH / 32;
constexpr int kTmaDimMax = 2048;            // longest rows (floats) staged through shared-memory slots

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

// Bounded wait for the phase with the given parity; false on expiry.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity)
{
    const uint32_t a = smem_u32(bar);
    for (uint32_t i = 0; i < WAIT_LIMIT; ++i) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(a), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}

// bytes (a multiple of 16) from global src (16-byte aligned) into shared dst
// (16-byte aligned), completion counted on bar, which expects them.
__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// Dynamic shared memory of the slot routine: the query row, the warps' slots,
// the in-band candidates, their keys, the slots' mbarriers.
struct RescoreSmem {
    size_t q, slots, cand, key, bar, bytes;
    __host__ __device__ RescoreSmem(int dim_pad, int spw, int cmax)
    {
        const size_t row = (size_t)dim_pad * 4;
        q = 0;
        slots = q + row;
        cand = slots + (size_t)kWarps * spw * row;
        int p2 = 1;
        while (p2 < cmax) p2 <<= 1;          // the keys' sort pads to a power of two
        key = cand + (((size_t)cmax * 4 + 7) / 8) * 8;
        bar = key + (size_t)p2 * 8;
        bytes = bar + (size_t)kWarps * spw * 8;
    }
};

// The R best of the n in-band keys (all distinct) into oi / oc in rank
// order, -1 / 0 past them.  Up to 256 keys: each one's rank counted against
// the others (a count stops once it reaches R: that key is not kept); more: a
// bitonic sort of the keys padded with zeros to a power of two (key holds
// that many slots).
__device__ __forceinline__ void rank_out(uint64_t *key, int n, int R, int32_t *__restrict__ oi,
                                         float *__restrict__ oc, int32_t out_stride)
{
    const int tid = threadIdx.x;
    if (n <= 256) {
        for (int i = tid; i < n; i += TH) {
            const uint64_t k = key[i];
            int c = 0;
            for (int j = 0; j < n && c < R; ++j) c += key[j] > k ? 1 : 0;
            if (c < R && c < out_stride) {
                oi[c] = (int32_t)(0xffffffffu - (uint32_t)(k & 0xffffffffu));
                if (oc) oc[c] = key_value((uint32_t)(k >> 32));
            }
        }
    } else {
        int P = 1;
        while (P < n) P <<= 1;
        for (int i = n + tid; i < P; i += TH) key[i] = 0ull;
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
        for (int i = tid; i < R && i < n && i < out_stride; i += TH) {
            oi[i] = (int32_t)(0xffffffffu - (uint32_t)(key[i] & 0xffffffffu));
            if (oc) oc[i] = key_value((uint32_t)(key[i] >> 32));
        }
    }
    for (int i = min(n, R) + tid; i < out_stride; i += TH) {
        oi[i] = -1;
        if (oc) oc[i] = 0.f;
    }
}

// One row through shared-memory slots: the C candidates cr (values cv,
// nullable) against the unit row q (global, dim_pad floats) -> the R best in
// rank order into oi / oc.  SPW slots per warp.
__device__ void rescore_row_slots(const float *__restrict__ q, int32_t dim_pad, const float *__restrict__ D32,
                                  const int32_t *__restrict__ cr, const float *__restrict__ cv, float band, int32_t C,
                                  int32_t R, int32_t *__restrict__ oi, float *__restrict__ oc, int32_t out_stride,
                                  int32_t n_obj, int spw, int cmax, int32_t *__restrict__ err)
{
    extern __shared__ __align__(128) uint8_t sm[];
    const RescoreSmem L(dim_pad, spw, cmax);
    float4 *q4 = reinterpret_cast<float4 *>(sm + L.q);
    float *slots = reinterpret_cast<float *>(sm + L.slots);
    int32_t *cand = reinterpret_cast<int32_t *>(sm + L.cand);
    uint64_t *key = reinterpret_cast<uint64_t *>(sm + L.key);
    uint64_t *bar = reinterpret_cast<uint64_t *>(sm + L.bar);
    __shared__ int s_n;
    __shared__ int s_fail;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nv = dim_pad / 4;
    const uint32_t row_bytes = (uint32_t)dim_pad * 4u;
    if (tid == 0) {
        s_n = 0;
        s_fail = 0;
        for (int i = 0; i < kWarps * spw; ++i) mbar_init(&bar[i], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    const float4 *src = reinterpret_cast<const float4 *>(q);
    for (int i = tid; i < nv; i += TH) q4[i] = src[i];
    __syncthreads();
    // the in-band candidates, compacted (their order is free: keys are ranked by counting)
    const float thr = cv ? cv[R - 1] - band : 0.f;
    for (int c0 = warp * 32; c0 < C; c0 += TH) {
        const int c = c0 + lane;
        // (an index outside the scene is never copied: such a candidate is dropped)
        const bool in = c < C && !(cv && cv[c] < thr) && cr[c] >= 0 && cr[c] < n_obj;
        const uint32_t m = __ballot_sync(0xffffffffu, in);
        int base = 0;
        if (lane == 0 && m) base = atomicAdd(&s_n, __popc(m));
        base = __shfl_sync(0xffffffffu, base, 0);
        if (in) cand[base + __popc(m & ((1u << lane) - 1u))] = cr[c];
    }
    __syncthreads();
    const int n = s_n;
    // warp w takes candidates w, w + W, ...; its i-th goes to its slot i % spw
    float *mine = slots + (size_t)warp * spw * dim_pad;
    uint64_t *mbar = bar + warp * spw;
    if (lane == 0)
        for (int k = 0; k < spw; ++k) {
            const int j = warp + kWarps * k;
            if (j < n) bulk_load(mine + (size_t)k * dim_pad, D32 + (int64_t)cand[j] * dim_pad, row_bytes, &mbar[k]);
        }
    bool ok = true;
    int issued = min(spw, (n - warp + kWarps - 1) / kWarps), done = 0;
    for (int i = 0;; ++i) {
        const int j = warp + kWarps * i;
        if (j >= n) break;
        const int k = i % spw;
        // (the lanes agree: a lane that gave up makes the whole warp give up)
        if (!__all_sync(0xffffffffu, mbar_wait(&mbar[k], (uint32_t)(i / spw) & 1u))) {
            ok = false;
            break;
        }
        const float4 *d4 = reinterpret_cast<const float4 *>(mine + (size_t)k * dim_pad);
        float a = 0.f;
        for (int v = lane; v < nv; v += 32) {
            const float4 x = d4[v], y = q4[v];
            a = fmaf(y.x, x.x, a);
            a = fmaf(y.y, x.y, a);
            a = fmaf(y.z, x.z, a);
            a = fmaf(y.w, x.w, a);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
        ++done;
        __syncwarp();     // every lane has read the slot
        if (lane == 0) {
            const int jn = j + kWarps * spw;
            if (jn < n) {
                bulk_load(mine + (size_t)k * dim_pad, D32 + (int64_t)cand[jn] * dim_pad, row_bytes, &mbar[k]);
                ++issued;
            }
            const int32_t e = cand[j];
            key[j] = ((uint64_t)order_key(a) << 32) | (uint64_t)(0xffffffffu - (uint32_t)e);
        }
        issued = __shfl_sync(0xffffffffu, issued, 0);
    }
    if (!ok) {
        // a copy did not arrive: record it, wait (bounded) for this warp's
        // copies still in flight, which target its slots, and give up the row
        if (lane == 0) {
            atomicOr(err, kErrTimeout);
            s_fail = 1;
            for (int i = done; i < issued; ++i) mbar_wait(&mbar[i % spw], (uint32_t)(i / spw) & 1u);
        }
    }
    __syncthreads();
    if (s_fail) {
        for (int i = tid; i < out_stride; i += TH) {
            oi[i] = -1;
            if (oc) oc[i] = 0.f;
        }
        return;
    }
    rank_out(key, n, R, oi, oc, out_stride);
}

// One row, loads from global memory: the C candidates cr (values cv, nullable) against the unit row q
// (global, dim_pad floats) -> the R best in rank order into oi / oc.
__device__ __forceinline__ void rescore_row_ldg(const float *__restrict__ q, int32_t dim_pad,
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

// Grouped rescore: block -> (piece, row) through the piece table; SLOTS:
// the rows go through spw shared-memory slots per warp, else global loads.
template <bool SLOTS>
__global__ void __launch_bounds__(TH)
rescore_grouped_kernel(const Piece *__restrict__ pieces, int32_t n_pieces, const float *__restrict__ Q32,
                       int32_t dim_pad, const int32_t *__restrict__ bsel_t, const float *__restrict__ bsel_tv,
                       int32_t cstride_t, const int32_t *__restrict__ bsel_l, const float *__restrict__ bsel_lv,
                       int32_t cstride_l, float band, int32_t *__restrict__ tsel_idx, float *__restrict__ tsel_cos,
                       int32_t stride_t, int32_t *__restrict__ lsel_idx, int32_t stride_l, int spw, int cmax,
                       int32_t *__restrict__ err)
{
    const int64_t r = blockIdx.x;
    const Piece pc = pieces[find_piece(pieces, n_pieces, r, [](const Piece &x) { return x.row_begin; })];
    const int i = (int)(r - pc.row_begin);
    const float *q = Q32 + (pc.q_row0 + i) * (int64_t)dim_pad;
    const bool tgt = i < pc.ntr;
    const int64_t l = pc.l_row0 + (i - pc.ntr);
    const int64_t co = tgt ? (pc.t_row0 + i) * (int64_t)cstride_t : l * (int64_t)cstride_l;
    const int32_t *cr = (tgt ? bsel_t : bsel_l) + co;
    const float *vals = tgt ? bsel_tv : bsel_lv;
    const float *cv = vals ? vals + co : nullptr;
    const int32_t C = tgt ? pc.fkeep_t : pc.fkeep_l, R = tgt ? pc.R : pc.klm;
    int32_t *oi = tgt ? tsel_idx + (pc.t_row0 + i) * (int64_t)stride_t : lsel_idx + l * (int64_t)stride_l;
    float *oc = tgt && tsel_cos ? tsel_cos + (pc.t_row0 + i) * (int64_t)stride_t : nullptr;
    const int32_t out = tgt ? stride_t : stride_l;
    if constexpr (SLOTS)
        rescore_row_slots(q, dim_pad, pc.d32, cr, cv, band, C, R, oi, oc, out, pc.n_obj, spw, cmax, err);
    else
        rescore_row_ldg(q, dim_pad, pc.d32, cr, cv, band, C, R, oi, oc, out);
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
                                   int32_t stride_l, int32_t *err, cudaStream_t s)
{
    if (total_rows <= 0) return cudaSuccess;
    if (n_pieces < 1 || total_rows > 0x7fffffff || dim_pad % 4 != 0 || cstride_t > SORT_MAX || cstride_l > SORT_MAX ||
        !err)
        return cudaErrorInvalidValue;
    // slots per warp: the count that keeps the most row copies in flight per
    // SM (resident CTAs x warps x slots; 228 KB of shared memory per SM, 1 KB
    // of it reserved per CTA); rows longer than kTmaDimMax floats take the
    // global-load routine
    const int cmax = cstride_t > cstride_l ? cstride_t : cstride_l;
    int spw = 0;
    if (dim_pad <= kTmaDimMax) {
        static const int regs = [] {
            cudaFuncAttributes a{};
            return cudaFuncGetAttributes(&a, rescore_grouped_kernel<true>) == cudaSuccess ? a.numRegs : 64;
        }();
        const int by_regs = 65536 / (((regs + 7) / 8 * 8) * TH), by_threads = 2048 / TH;
        int best = 0;
        for (int k = 1; k <= 4; ++k) {
            const size_t b = RescoreSmem(dim_pad, k, cmax).bytes + 256;
            if (b > 227 * 1024) break;
            int ctas = (int)((228 * 1024) / (b + 1024));
            ctas = ctas < by_regs ? ctas : by_regs;
            ctas = ctas < by_threads ? ctas : by_threads;
            if (ctas * kWarps * k > best) {
                best = ctas * kWarps * k;
                spw = k;
            }
        }
    }
    const size_t smem = spw > 0 ? RescoreSmem(dim_pad, spw, cmax).bytes : (size_t)dim_pad * sizeof(float);
    auto kern = spw > 0 ? rescore_grouped_kernel<true> : rescore_grouped_kernel<false>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    kern<<<(unsigned)total_rows, TH, smem, s>>>(pieces, n_pieces, Q32, dim_pad, bsel_t, bsel_tv, cstride_t, bsel_l,
                                                bsel_lv, cstride_l, band, tsel_idx, tsel_cos, stride_t, lsel_idx,
                                                stride_l, spw, cmax, err);
    return cudaGetLastError();
}

}  // namespace farm
