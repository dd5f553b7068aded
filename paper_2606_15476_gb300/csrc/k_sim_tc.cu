// k_sim_tc.cu -- descriptor similarity on the 5th-generation tensor cores
// (App. D.2 step 3: the cosine of every query row against every object).
//
// Three arithmetic modes share one kernel template:
//  * FP32-accurate, three FP16 products with a scaled residual:
//      S[r, j] = <q_r, d_j> ~= q_hi.d_hi + 2^-11 (q_hi.d_lo + q_lo.d_hi)
//  * BF16: S[r, j] ~= <bf16(q_r), bf16(d_j)> with FP32 accumulation;
//  * FP8-E4M3 with per-row scales: S[r, j] ~= s_r t_j <e4m3(q_r/s_r), e4m3(d_j/t_j)>,
//    the scales applied in the epilogue.
//  The last two are the first stage of the reduced-precision paths (their
//  borderline candidates are re-scored in FP32 afterwards).
//
// FP32-accurate mode (the split of Ootomo and Yokota, "Recovering single
// precision accuracy from Tensor Cores while surpassing the FP32 theoretical
// peak performance", IJHPCA 2022): with x_hi = FP16(x) and
// x_lo = FP16(2^11 (x - x_hi)) prepared by the normalisation kernel, each
// operand keeps 22 significant bits; the dropped x_lo*y_lo term and the
// rounding of x_lo are each about 2^-22 of |x*y|.  The 2^11 scale keeps the
// residual in FP16's normal range.  The tensor cores' FP32 accumulation
// truncates: every MMA step adds an error of up to one unit in the last place
// of the running sum, so the large products q_hi.d_hi accumulate in one
// tensor-memory (TMEM) accumulator and the two scaled correction products in
// a second one; the epilogue adds 2^-11 times the second to the first in IEEE
// FP32.  FP16 products run at twice the TF32 rate and the operands take half
// the bytes of a TF32 split.
//
// Kernel organisation (persistent: one CTA per SM -- 192 threads, or 320
// with eight epilogue warps -- walks the 128 x BN tiles of S; in a CTA pair
// the two CTAs of a cluster compute one 256 x 256 tile together):
//   warp 0      TMA producer: for each K slice (32 FP16 values, 64-byte swizzle,
//               four tiles q_hi, q_lo, d_hi, d_lo; or 64 BF16 / 128 FP8 values,
//               128-byte swizzle, two tiles q, d) fills one pipeline stage,
//               signalling a "full" mbarrier with the byte count (a pair: both
//               CTAs' copies count on the even CTA's barrier);
//   warp 1      allocates TMEM (main and correction 128 x 256 FP32
//               accumulators in the FP32-accurate mode, two alternating tile
//               accumulators otherwise); one thread issues, per K slice,
//               2 K-steps x 3 products of tcgen05.mma.kind::f16 with FP16
//               operands (M=128, or 256 for a pair; N=256, K=16), or 4 K-steps
//               of kind::f16 (BF16) / kind::f8f6f4 (E4M3), and tcgen05.commit
//               to the stage's "empty" mbarrier, finally to the "accumulator
//               ready" mbarrier;
//   warps 2-5   epilogue (warps 2-9 when eight: two per TMEM lane quarter,
//               each taking half of the tile's columns): tcgen05.ld 32 lanes
//               x 32 columns at a time, each 32 x 32 block staged through
//               shared memory so that stores write whole row segments of S
//               (bounds-checked), the group maxima likewise, then release the
//               accumulator.  FP32-accurate mode at 256-object tiles (eight
//               warps) folds the correction into registers and releases both
//               accumulators before it stores or compares, so the next tile's
//               MMAs wait only for the TMEM loads; FP8 tiles take eight warps
//               too.
// Stages of 48 KB (32 KB in a pair) within 192 KB, and no more than the
// shared memory left beside 4 KB of epilogue staging per epilogue warp (and
// the fused selection's candidate slots).  Every mbarrier wait is bounded: on expiry the kernel raises the
// error flag, stops issuing work, waits (bounded) for the copies it issued,
// frees its TMEM and returns.
#include <algorithm>

#include <cuda.h>
#include <cudaTypedefs.h>

#include "farm_internal.h"

namespace farm {
namespace {

constexpr int BM = kSimTileM;
constexpr int STAGE_BUDGET = 192 * 1024;     // shared memory for the operand pipeline
constexpr uint32_t WAIT_LIMIT = 1u << 24;    // try_wait polls before giving up (about a second)
constexpr int GROUP_M = 8;                   // tile raster: 8 cluster rows share each column tile
constexpr float RESID_SCALE_INV = 1.f / 2048.f;   // the residual operands carry a factor 2^11

// Per-mode element layout of the operand rows of a K slice.
template <int MODE>
struct Elem;
template <>
struct Elem<kSimF16x3> {                     // three-term FP16 with scaled residuals
    static constexpr int BK = 32;            // FP16 elements per K slice (64-byte rows)
    static constexpr int ROW_BYTES = 64;
    static constexpr int KSTEPS = 2;         // 16 FP16 values (32 bytes) per MMA
    static constexpr bool SPLIT = true;      // hi and lo tiles of each operand
    static constexpr uint64_t LAYOUT = 4;    // 64-byte swizzle
    static constexpr uint32_t SBO = 512;     // 8 rows x 64 bytes
};
template <>
struct Elem<kSimBf16> {                      // BF16
    static constexpr int BK = 64;            // BF16 elements per K slice (128-byte rows)
    static constexpr int ROW_BYTES = 128;
    static constexpr int KSTEPS = 4;         // 16 BF16 values (32 bytes) per MMA
    static constexpr bool SPLIT = false;
    static constexpr uint64_t LAYOUT = 2;    // 128-byte swizzle
    static constexpr uint32_t SBO = 1024;    // 8 rows x 128 bytes
};
template <>
struct Elem<kSimFp8> {                       // FP8 E4M3
    static constexpr int BK = 128;           // FP8 elements per K slice (128-byte rows)
    static constexpr int ROW_BYTES = 128;
    static constexpr int KSTEPS = 4;         // 32 FP8 values (32 bytes) per MMA
    static constexpr bool SPLIT = false;
    static constexpr uint64_t LAYOUT = 2;    // 128-byte swizzle
    static constexpr uint32_t SBO = 1024;    // 8 rows x 128 bytes
};

// A tile configuration: BN objects per tile, CM CTAs per cluster (1, or 2
// for a pair); PAIR: the two CTAs of a cluster compute one 256 x BN tile with
// two-SM MMAs (cta_group::2), each holding its 128 rows of A and half of B.
// Every CTA loads its own operand tiles: no copy is delivered to several CTAs.
// EMIT_: the fused selection's epilogue, whose candidate slots (32 KB) take
// the place of one pipeline stage.  Folded FP32-accurate tiles (one tile in
// TMEM) get eight epilogue warps, two per TMEM lane quarter, each taking half
// of the tile's columns into registers (16 candidate slots per thread) and
// releasing the accumulators before it compares or stores: the next tile's
// main products wait only for the TMEM loads.  FP8 tiles get eight warps too.
template <int MODE, int BN_, int CM_, bool PAIR_ = false, bool EMIT_ = false>
struct Cfg {
    using E = Elem<MODE>;
    static constexpr int BN = BN_;
    static constexpr int CM = CM_;
    static constexpr int OPS = E::SPLIT ? 2 : 1;                // operand copies (hi, lo)
    static constexpr int A_BYTES = BM * E::ROW_BYTES;
    static constexpr int B_BYTES = BN_ * E::ROW_BYTES;
    static constexpr int B_PART = B_BYTES / CM_;                // this CTA's share of a B tile
    static constexpr int B_SMEM = PAIR_ ? B_PART : B_BYTES;     // B bytes a stage holds in this CTA
    static constexpr int STAGE_BYTES = OPS * (A_BYTES + B_SMEM);
    static constexpr int ACC_COLS = OPS * BN_;                  // TMEM columns of one tile's accumulators
    static constexpr int NACC = 512 / ACC_COLS >= 2 ? 2 : 1;    // tiles in flight in TMEM
    static constexpr bool FOLD = E::SPLIT && NACC == 1;         // the correction is folded into the main accumulator
    // epilogue warps, two or one per TMEM lane quarter: eight for the 256-object
    // tiles whose epilogue bounds the tile (FP32-accurate tiles, which hold
    // TMEM alone; FP8, whose MMAs are few); BF16 tiles overlap four warps'
    // epilogue with the next tile's MMAs
    static constexpr int EPI_WARPS = BN_ == 256 && (FOLD || MODE == kSimFp8) ? 8 : 4;
    static constexpr int THREADS = 64 + 32 * EPI_WARPS;         // + the producer and MMA warps
    static constexpr int EMIT_SLOTS = 32 * 4 / EPI_WARPS;       // candidate words per epilogue thread
    static constexpr int EMIT_BYTES = EMIT_ ? EPI_WARPS * 32 * EMIT_SLOTS * 8 : 0;
    static constexpr int STAGING_BYTES = EPI_WARPS * 32 * 32 * 4;      // epilogue: one 32 x 32 FP32 block per warp
    static constexpr int SCALE_BYTES = MODE == kSimFp8 ? EPI_WARPS * BN_ * 4 : 0;   // FP8: a tile's column scales per warp
    static constexpr int FIXED_BYTES = 1024 /*align*/ + 256 /*barriers*/ + STAGING_BYTES + SCALE_BYTES + EMIT_BYTES;
    static constexpr int BUDGET = STAGE_BUDGET < 227 * 1024 - FIXED_BYTES ? STAGE_BUDGET : 227 * 1024 - FIXED_BYTES;
    static constexpr int STAGES = BUDGET / STAGE_BYTES < 8 ? BUDGET / STAGE_BYTES : 8;
    static constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + FIXED_BYTES;
    static_assert(SMEM_BYTES <= 227 * 1024, "shared memory per CTA");
    static_assert(BN_ % 128 == 0 && BN_ <= 256, "tile width");
    static_assert(STAGES >= 3, "pipeline depth");
    static_assert(BN_ / CM_ >= 8 && (B_PART % 1024) == 0, "B share must keep the swizzle atoms whole");
    static_assert(!PAIR_ || (CM_ == 2 && BN_ == 256), "CTA pairs: clusters of two, 256-object tiles");
    static_assert(PAIR_ || CM_ == 1, "clusters of two only as CTA pairs");
};

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
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

// One non-blocking test of the phase with the given parity.
__device__ __forceinline__ bool mbar_test(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, uint64_t *bar, int c0, int c1)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];"
        ::"r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(c0), "r"(c1)
        : "memory");
}

__device__ __forceinline__ uint32_t cluster_rank()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

// Every thread of every CTA of the cluster (release / acquire).
__device__ __forceinline__ void cluster_sync()
{
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// Shared-memory matrix descriptor of a K-major operand tile with rows of
// ROW_BYTES swizzled in 8-row core groups SBO bytes apart; version 1.  The
// leading byte offset is unused for swizzled K-major layouts.
template <int MODE>
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);              // start address
    d |= (uint64_t)(Elem<MODE>::SBO >> 4) << 32;            // stride byte offset
    d |= (uint64_t)1 << 46;                                 // descriptor version
    d |= Elem<MODE>::LAYOUT << 61;                          // swizzle mode
    return d;
}

// Instruction descriptors: D = F32, A and B K-major, M = m (128, or 256 for
// a CTA pair), N = n; operand format FP16 (0, kind::f16), BF16 (1,
// kind::f16) or E4M3 (0, kind::f8f6f4).
__host__ __device__ constexpr uint32_t idesc(uint32_t ab_format, int n, int m)
{
    return (1u << 4)                      // D format F32
           | (ab_format << 7)             // A format
           | (ab_format << 10)            // B format
           | ((uint32_t)(n >> 3) << 17)   // N / 8
           | ((uint32_t)(m >> 4) << 24);  // M / 16
}

// One MMA of the mode's kind (FP16 and BF16 operands: kind::f16; E4M3:
// kind::f8f6f4), D (+)= A B^T into TMEM; PAIR: a two-SM MMA (M = 256) over
// both CTAs' shared-memory halves and TMEM, issued by the even CTA.
template <int MODE, int BN_, bool PAIR>
__device__ __forceinline__ void mma(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t accumulate)
{
    constexpr uint32_t id = idesc(MODE == kSimBf16 ? 1u : 0u, BN_, PAIR ? 2 * BM : BM);
    if (MODE == kSimFp8 && !PAIR) {
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "setp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}"
            ::"r"(d_tmem), "l"(a_desc), "l"(b_desc), "r"(id), "r"(accumulate));
    } else if (MODE == kSimFp8) {
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "setp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::2.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}"
            ::"r"(d_tmem), "l"(a_desc), "l"(b_desc), "r"(id), "r"(accumulate));
    } else if (!PAIR) {
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "setp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
            ::"r"(d_tmem), "l"(a_desc), "l"(b_desc), "r"(id), "r"(accumulate));
    } else {
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "setp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n\t}"
            ::"r"(d_tmem), "l"(a_desc), "l"(b_desc), "r"(id), "r"(accumulate));
    }
}

__device__ __forceinline__ void mma_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

// 32 columns of the warp's 32 TMEM lanes (lane = row), without the wait.
__device__ __forceinline__ void tmem_ld32_issue(uint32_t taddr, uint32_t (&r)[32])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
          "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
          "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
          "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32])
{
    uint32_t r[32];
    tmem_ld32_issue(taddr, r);
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// Two 32-column loads behind one wait.
__device__ __forceinline__ void tmem_ld32_pair(uint32_t ta, uint32_t tb, float (&v)[32], float (&w)[32])
{
    uint32_t r[32], q[32];
    tmem_ld32_issue(ta, r);
    tmem_ld32_issue(tb, q);
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) {
        v[i] = __uint_as_float(r[i]);
        w[i] = __uint_as_float(q[i]);
    }
}

// The pair's commit: arrives on the mbarrier at the offset of `bar` in both
// CTAs once the two-SM MMAs issued so far have completed.
__device__ __forceinline__ void mma_commit_pair(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;"
                 ::"r"(smem_u32(bar)), "h"((uint16_t)3)
                 : "memory");
}

// Cluster address of the object at this CTA's shared-memory address `saddr`
// in the CTA of the given cluster rank.
__device__ __forceinline__ uint32_t cluster_addr(uint32_t saddr, uint32_t rank)
{
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(saddr), "r"(rank));
    return r;
}

// A TMA load into this CTA's shared memory whose completion is counted on an
// mbarrier of either CTA of the pair (bar: cluster address).
__device__ __forceinline__ void tma_load_2d_pair(void *dst, const CUtensorMap *map, uint32_t bar, int c0, int c1)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes.cta_group::2"
        " [%0], [%1, {%3, %4}], [%2];"
        ::"r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(bar), "r"(c0), "r"(c1)
        : "memory");
}

// Arrive on an mbarrier of another CTA of the cluster (cluster address).
__device__ __forceinline__ void mbar_arrive_remote(uint32_t bar)
{
    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(bar) : "memory");
}

// Store 32 consecutive columns of the warp's 32 TMEM lanes (one per thread).
__device__ __forceinline__ void tmem_st32(uint32_t taddr, const float (&v)[32])
{
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], "
        "{%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,"
        "%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};"
        ::"r"(taddr), "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
          "r"(__float_as_uint(v[3])), "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])),
          "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])), "r"(__float_as_uint(v[8])),
          "r"(__float_as_uint(v[9])), "r"(__float_as_uint(v[10])), "r"(__float_as_uint(v[11])),
          "r"(__float_as_uint(v[12])), "r"(__float_as_uint(v[13])), "r"(__float_as_uint(v[14])),
          "r"(__float_as_uint(v[15])), "r"(__float_as_uint(v[16])), "r"(__float_as_uint(v[17])),
          "r"(__float_as_uint(v[18])), "r"(__float_as_uint(v[19])), "r"(__float_as_uint(v[20])),
          "r"(__float_as_uint(v[21])), "r"(__float_as_uint(v[22])), "r"(__float_as_uint(v[23])),
          "r"(__float_as_uint(v[24])), "r"(__float_as_uint(v[25])), "r"(__float_as_uint(v[26])),
          "r"(__float_as_uint(v[27])), "r"(__float_as_uint(v[28])), "r"(__float_as_uint(v[29])),
          "r"(__float_as_uint(v[30])), "r"(__float_as_uint(v[31]))
        : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Cluster tile id -> this CTA's (first row, first column).  A cluster tile is
// CM vertically adjacent row tiles (CTA rank r takes the r-th) of one column
// tile; under the grouped raster GROUP_M cluster rows share each column tile
// so a descriptor tile is read from HBM about once per group.
template <int BN_, int CM_>
__device__ __forceinline__ void tile_origin(int tile, int m_super, int n_tiles, uint32_t rank, int &m0, int &n0)
{
    const int per_group = GROUP_M * n_tiles;
    const int g = tile / per_group;
    const int first_m = g * GROUP_M;
    // (a tile past the piece, which a correct tile count never gives, lands
    // beyond its last row: loads read the zero fill, the epilogue writes nothing)
    const int gm = max(1, min(GROUP_M, m_super - first_m));
    const int in_g = tile - g * per_group;
    m0 = ((first_m + in_g % gm) * CM_ + (int)rank) * BM;
    n0 = (in_g / gm) * BN_;
}

// Persistent: cluster c (one CTA, or a CTA pair) walks cluster tiles c,
// c + (number of clusters), ....  A stage is full when the CTA's A tile and
// its B tile (a pair: both CTAs' A tiles and B halves, counted on the even
// CTA's barrier) have landed, and free again when the MMAs that read it have
// completed.  The shared-memory pipeline runs on across tiles.  When two
// tiles' accumulators fit the 512 TMEM columns (BF16 and FP8; FP16x3 at
// 128-object tiles, whose main and correction accumulators take 256 columns)
// the epilogue of one tile overlaps the MMAs of the next (acc_full /
// acc_empty mbarriers); FP16x3 at 256-object tiles folds the correction
// accumulator first so that the next tile's correction products overlap the
// stores, while the producer already prefetches that tile's first stages.
// A launch covers either one problem (`single`, its B maps map_d0 / map_d1)
// or, GROUPED, the pieces of a device table: blocks of query rows against
// different scenes, with their B maps in device memory, numbered by cluster
// tile (tile_begin) so that every role finds its piece by binary search.
// Maps (FP16x3 mode): q_hi, q_lo, d_hi, d_lo.  (BF16, FP8 modes): q, d, and
// the second of each pair is unused.  scale_q: per-row scales of the query
// rows, pieces' scale_d: per-object scales (FP8 mode only).
template <bool GROUPED>
__device__ __forceinline__ GemmPiece piece_of(int tile, const GemmPiece *pieces, int n_pieces,
                                              const GemmPiece &single)
{
    if (!GROUPED) return single;
    int lo = 0, hi = n_pieces - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (pieces[mid].tile_begin <= tile) lo = mid;
        else hi = mid - 1;
    }
    return pieces[lo];
}

// This CTA's tile of cluster tile `tile` within piece pc: first row (local
// to the piece), first object column n0 and first stored column c0 (they
// differ for the compacted sample tiles).
template <int BN_, int CM_>
__device__ __forceinline__ void piece_tile(const GemmPiece &pc, int tile, uint32_t rank, int &m0, int &n0, int &c0)
{
    const int m_tiles = (pc.rows + BM - 1) / BM;
    const int n_tiles = (int)col_tiles(pc.n, BN_, pc.col_mode, pc.col_stride);
    tile_origin<BN_, CM_>(tile - pc.tile_begin, (m_tiles + CM_ - 1) / CM_, n_tiles, rank, m0, c0);
    n0 = (int)col_tile_of(c0 / BN_, pc.col_mode, pc.col_stride) * BN_;
}

__device__ __forceinline__ uint32_t order_key(float f)
{
    const uint32_t u = __float_as_uint(f + 0.0f);   // -0 -> +0
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

__device__ __forceinline__ float key_value(uint32_t k)
{
    const uint32_t u = (k & 0x80000000u) ? (k & 0x7fffffffu) : ~k;
    return __uint_as_float(u);
}

// Store SL float4 values per row of the warp's 32 rows (lane = row) to
// dst + row * stride through the warp's shared-memory block (slots
// XOR-swizzled by row), so that a store instruction writes whole row segments
// of SL * 16 bytes; rows >= rows_left are skipped.
template <int SL>
__device__ __forceinline__ void store_rows_staged(float4 *blk, const float4 (&val)[SL], int lane, float *dst,
                                                  int64_t stride, int64_t rows_left)
{
#pragma unroll
    for (int j = 0; j < SL; ++j) blk[lane * SL + (j ^ (lane & (SL - 1)))] = val[j];
    __syncwarp();
#pragma unroll
    for (int it = 0; it < SL; ++it) {
        const int q = it * 32 + lane, rr = q / SL, sl = q % SL;
        const float4 x = blk[rr * SL + (sl ^ (rr & (SL - 1)))];
        if (rr < rows_left) *reinterpret_cast<float4 *>(dst + rr * stride + sl * 4) = x;
    }
    __syncwarp();
}

template <int MODE, int BN_, int CM_, bool GROUPED, bool PAIR, bool EMIT = false>
__global__ void __launch_bounds__((Cfg<MODE, BN_, CM_, PAIR, EMIT>::THREADS), 1)
sim_tc_kernel(const __grid_constant__ CUtensorMap map_q0, const __grid_constant__ CUtensorMap map_q1,
              const __grid_constant__ CUtensorMap map_d0, const __grid_constant__ CUtensorMap map_d1,
              const GemmPiece *__restrict__ pieces, int32_t n_pieces, const GemmPiece single,
              float *__restrict__ S, float *__restrict__ tops, int32_t k_slices, int32_t total,
              const float *__restrict__ scale_q, int32_t *err, const FuseEmit emit)
{
    using C = Cfg<MODE, BN_, CM_, PAIR, EMIT>;
    using M = Elem<MODE>;
    constexpr bool TWO_OPERAND_TILES = !M::SPLIT;
    constexpr int B_SMEM = C::B_SMEM;
    constexpr int NACC = C::NACC;
    constexpr int STAGES = C::STAGES;
    constexpr int STAGE_BYTES = C::STAGE_BYTES;
    constexpr int BN = BN_, CM = CM_;
    constexpr int ACC_CORR = BN_;            // correction accumulator: the columns after the main one
    // FP32-accurate mode with one tile in TMEM: the epilogue first folds the
    // correction into the main accumulator in TMEM and frees the correction
    // columns, so the next tile's correction products (two thirds of its
    // MMAs) run while the main accumulator is drained to S (EMIT: compared
    // with the rows' thresholds).
    constexpr bool FOLD = C::FOLD;
    static_assert(!EMIT || GROUPED, "the fused selection runs grouped launches");
    constexpr uint32_t TMEM_ALLOC = 512;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + STAGES * STAGE_BYTES);
    uint64_t *empty = full + STAGES;
    uint64_t *acc_full = empty + STAGES;
    uint64_t *acc_empty = acc_full + 2;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(acc_empty + 2);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
    float *staging = reinterpret_cast<float *>(smem + STAGES * STAGE_BYTES + 256);
    float *tile_scales = staging + C::EPI_WARPS * 32 * 32;    // FP8 mode: [epilogue warps][BN]
    // EMIT: [epilogue warps][32 lanes][EMIT_SLOTS] candidate words
    uint64_t *emit_slots = reinterpret_cast<uint64_t *>(reinterpret_cast<uint8_t *>(tile_scales) + C::SCALE_BYTES);
    uint64_t *corr_free = acc_empty + 1;      // FOLD: the correction columns are free (tile accumulators: one)

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t rank = cluster_rank();
    const int cluster_id = blockIdx.x / CM, n_clusters = gridDim.x / CM;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            // one commit from the MMA issuer (a pair: the even CTA's, arriving in both CTAs)
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&acc_full[b], 1);
            mbar_init(&acc_empty[b], (PAIR ? 2 : 1) * C::EPI_WARPS);   // one arrival per epilogue warp (of both CTAs of a pair)
        }
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        // a pair: one warp of each CTA allocates collectively (the same columns in both)
        if (PAIR) {
            asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;"
                         ::"r"(smem_u32(tmem_slot)), "r"(TMEM_ALLOC));
            asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;");
        } else {
            asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                         ::"r"(smem_u32(tmem_slot)), "r"(TMEM_ALLOC));
            asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    cluster_sync();    // a pair: both CTAs' mbarriers are initialised before the peer's copies or commits reach them
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            uint32_t it = 0;
            for (int tile = cluster_id; tile < total && !*abort_flag; tile += n_clusters) {
                const GemmPiece pc = piece_of<GROUPED>(tile, pieces, n_pieces, single);
                int m0, n0, c0;
                piece_tile<BN_, CM_>(pc, tile, rank, m0, n0, c0);
                const int qa = (int)(pc.q_row0 + m0);     // A rows: the piece's rows in the operand arrays
                const CUtensorMap *bmap0 = GROUPED ? static_cast<const CUtensorMap *>(pc.bmap) : &map_d0;
                const CUtensorMap *bmap1 = GROUPED ? static_cast<const CUtensorMap *>(pc.bmap) + 1 : &map_d1;
                if (GROUPED && (reinterpret_cast<uintptr_t>(pc.bmap) & 63u)) {
                    // a tensor map must be 64-byte aligned: never hand the copy engine anything else
                    atomicOr(err, kErrPieceTable);
                    *abort_flag = 1;
                    break;
                }
                for (int kb = 0; kb < k_slices; ++kb, ++it) {
                    const int s = it % STAGES;
                    const uint32_t ph = (it / STAGES) & 1u;
                    if (!mbar_wait(&empty[s], ph ^ 1u) || *abort_flag) {
                        *abort_flag = 1;
                        break;
                    }
                    uint8_t *st = smem + s * STAGE_BYTES;
                    const int kx = kb * M::BK;
                    const int nb = n0 + (int)rank * (BN / CM);   // first B row of this CTA's share
                    if (PAIR) {
                        // both CTAs' copies count on the even CTA's "full" barrier, which
                        // expects the pair's bytes; each CTA holds its rows of A and its
                        // half of B at the same offsets
                        if (rank == 0) mbar_expect_tx(&full[s], 2 * STAGE_BYTES);
                        const uint32_t fb = cluster_addr(smem_u32(&full[s]), 0u);
                        if (TWO_OPERAND_TILES) {
                            tma_load_2d_pair(st, &map_q0, fb, kx, qa);
                            tma_load_2d_pair(st + C::A_BYTES, bmap0, fb, kx, nb);
                        } else {
                            tma_load_2d_pair(st, &map_q0, fb, kx, qa);
                            tma_load_2d_pair(st + C::A_BYTES, &map_q1, fb, kx, qa);
                            tma_load_2d_pair(st + 2 * C::A_BYTES, bmap0, fb, kx, nb);
                            tma_load_2d_pair(st + 2 * C::A_BYTES + B_SMEM, bmap1, fb, kx, nb);
                        }
                        continue;
                    }
                    mbar_expect_tx(&full[s], STAGE_BYTES);
                    if (TWO_OPERAND_TILES) {
                        tma_load_2d(st, &map_q0, &full[s], kx, qa);
                        tma_load_2d(st + C::A_BYTES, bmap0, &full[s], kx, nb);
                    } else {
                        tma_load_2d(st, &map_q0, &full[s], kx, qa);
                        tma_load_2d(st + C::A_BYTES, &map_q1, &full[s], kx, qa);
                        tma_load_2d(st + 2 * C::A_BYTES, bmap0, &full[s], kx, nb);
                        tma_load_2d(st + 2 * C::A_BYTES + C::B_BYTES, bmap1, &full[s], kx, nb);
                    }
                }
            }
            if (*abort_flag) {
                // let the copies already issued land before shared memory is released
                // (a pair's copies are counted on the even CTA's barriers)
                if (!PAIR || rank == 0)
                    for (uint32_t j = (it > (uint32_t)STAGES ? it - STAGES : 0u); j < it; ++j)
                        mbar_wait(&full[j % STAGES], (j / STAGES) & 1u);
                atomicOr(err, kErrTimeout);
            }
        }
    } else if (warp == 1) {
        if (lane == 0 && (!PAIR || rank == 0)) {     // a pair's MMAs are issued by its even CTA
            // the products of K slice kb from stage s: the main one (hi.hi, or the
            // only one) and / or the two correction products
            auto issue = [&](uint32_t acc, int kb, int s, bool main, bool corr) {
                const uint32_t st = smem_u32(smem + s * STAGE_BYTES);
                if (TWO_OPERAND_TILES) {
                    const uint32_t a = st, b = st + C::A_BYTES;
#pragma unroll
                    for (int kk = 0; kk < M::KSTEPS; ++kk) {
                        const uint32_t off = kk * 32;     // 32 bytes along K: 16 BF16 or 32 FP8 values
                        mma<MODE, BN_, PAIR>(acc, smem_desc<MODE>(a + off), smem_desc<MODE>(b + off),
                                             (kb | kk) != 0);
                    }
                } else {
                    const uint32_t a_hi = st, a_lo = st + C::A_BYTES;
                    const uint32_t b_hi = st + 2 * C::A_BYTES, b_lo = st + 2 * C::A_BYTES + B_SMEM;
#pragma unroll
                    for (int kk = 0; kk < M::KSTEPS; ++kk) {
                        const uint32_t off = kk * 32;     // 16 FP16 values = 32 bytes along K
                        const uint32_t first = (kb | kk) != 0;
                        if (main)
                            mma<MODE, BN_, PAIR>(acc, smem_desc<MODE>(a_hi + off), smem_desc<MODE>(b_hi + off),
                                                 first);
                        if (corr) {
                            mma<MODE, BN_, PAIR>(acc + ACC_CORR, smem_desc<MODE>(a_hi + off),
                                                 smem_desc<MODE>(b_lo + off), first);
                            mma<MODE, BN_, PAIR>(acc + ACC_CORR, smem_desc<MODE>(a_lo + off),
                                                 smem_desc<MODE>(b_hi + off), 1u);
                        }
                    }
                }
            };
            auto release = [&](int s) {
                if (PAIR) mma_commit_pair(&empty[s]);
                else mma_commit(&empty[s]);
            };
            uint32_t it = 0, tc = 0;
            for (int tile = cluster_id; tile < total && !*abort_flag; tile += n_clusters, ++tc) {
                const uint32_t buf = tc % NACC, use = tc / NACC;
                // FOLD: the correction columns are free after the previous tile's fold,
                // the main columns after its stores; otherwise both with the accumulator
                if (!mbar_wait(FOLD ? corr_free : &acc_empty[buf], (use & 1u) ^ 1u) || *abort_flag) {
                    *abort_flag = 1;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;");
                const uint32_t acc = tmem + buf * (uint32_t)C::ACC_COLS;
                // FOLD: until the main columns are free, slices get their correction
                // products only and keep their stage ("held"); at most STAGES of them,
                // since the producer refills a stage only once it is released
                bool main_ready = !FOLD;
                int held = 0, held_kb = 0;
                uint32_t held_it = 0;
                auto flush = [&]() {
                    for (int j = 0; j < held; ++j) {
                        const int sj = (int)((held_it + (uint32_t)j) % STAGES);
                        issue(acc, held_kb + j, sj, true, false);
                        release(sj);
                    }
                    held = 0;
                };
                for (int kb = 0; kb < k_slices; ++kb, ++it) {
                    const int s = it % STAGES;
                    const uint32_t ph = (it / STAGES) & 1u;
                    if (FOLD && !main_ready && held >= STAGES) {
                        if (!mbar_wait(&acc_empty[buf], (use & 1u) ^ 1u) || *abort_flag) {
                            *abort_flag = 1;
                            break;
                        }
                        asm volatile("tcgen05.fence::after_thread_sync;");
                        main_ready = true;
                        flush();
                    }
                    if (!mbar_wait(&full[s], ph) || *abort_flag) {
                        *abort_flag = 1;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;");
                    if (FOLD && !main_ready && mbar_test(&acc_empty[buf], (use & 1u) ^ 1u)) {
                        asm volatile("tcgen05.fence::after_thread_sync;");
                        main_ready = true;
                        flush();
                    }
                    issue(acc, kb, s, main_ready, true);
                    if (main_ready) {
                        release(s);
                    } else {
                        if (held == 0) {
                            held_kb = kb;
                            held_it = it;
                        }
                        ++held;
                    }
                }
                if (*abort_flag) break;
                if (FOLD && !main_ready) {
                    if (!mbar_wait(&acc_empty[buf], (use & 1u) ^ 1u) || *abort_flag) {
                        *abort_flag = 1;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;");
                    flush();
                }
                if (PAIR) mma_commit_pair(&acc_full[buf]);
                else mma_commit(&acc_full[buf]);
            }
            if (*abort_flag) atomicOr(err, kErrTimeout);
        }
    } else {
        // epilogue: warp w reads TMEM lanes 32*(w%4) .. +31 (with eight
        // epilogue warps, warps w and w + 4 take the two halves of the
        // columns).  Each 32-row x 32-column block passes through the warp's
        // shared-memory block (16-byte slots XOR-swizzled by row, conflict-free
        // both ways) so that every store instruction writes four whole 128-byte
        // row segments of S instead of 16 bytes in each of 32 rows.
        const int quad = warp & 3;
        constexpr int NCH = BN / 32 / (C::EPI_WARPS / 4);     // the warp's 32-column chunks
        const int cbase = ((warp - 2) >> 2) * NCH;             // its first chunk
        float4 *blk = reinterpret_cast<float4 *>(staging + (warp - 2) * 32 * 32);
        const int sub = lane >> 3, slot = lane & 7;    // read-back: row sub + 4i, 16-byte slot
        uint32_t tc = 0;
        for (int tile = cluster_id; tile < total; tile += n_clusters, ++tc) {
            const uint32_t buf = tc % NACC, use = tc / NACC;
            // EMIT: the row's threshold is read before the accumulator is waited for
            uint32_t tk = 0xffffffffu;
            if constexpr (EMIT) {
                const GemmPiece pt = piece_of<GROUPED>(tile, pieces, n_pieces, single);
                int tm0, tn0, tc0;
                piece_tile<BN_, CM_>(pt, tile, rank, tm0, tn0, tc0);
                const int64_t tr = (int64_t)tm0 + quad * 32 + lane;
                if (tr < pt.rows) tk = __ldg(emit.tau_key + pt.q_row0 + tr);
            }
            if (!mbar_wait(&acc_full[buf], use & 1u) || *abort_flag) {
                *abort_flag = 1;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;");
            // FOLD with eight epilogue warps: the warp's folded chunks stay in
            // registers and both accumulators are released at once, before the
            // compares or stores
            constexpr bool REGS = FOLD && C::EPI_WARPS == 8;
            float fv[REGS ? NCH : 1][32];
            if (FOLD) {
                // main += 2^-11 correction (in place, or into registers); then the
                // correction columns are free
                const uint32_t tb = tmem + ((uint32_t)(quad * 32) << 16);
                if constexpr (REGS) {
#pragma unroll
                    for (int cc = 0; cc < NCH; ++cc) {
                        const uint32_t ta = tb + (uint32_t)((cbase + cc) * 32);
                        float w[32];
                        tmem_ld32_pair(ta, ta + ACC_CORR, fv[cc], w);
#pragma unroll
                        for (int i = 0; i < 32; ++i) fv[cc][i] = fmaf(w[i], RESID_SCALE_INV, fv[cc][i]);
                    }
                } else {
#pragma unroll
                    for (int cc = 0; cc < NCH; ++cc) {
                        const int c = cbase + cc;
                        float v[32], w[32];
                        tmem_ld32(tb + (uint32_t)(c * 32), v);
                        tmem_ld32(tb + ACC_CORR + (uint32_t)(c * 32), w);
#pragma unroll
                        for (int i = 0; i < 32; ++i) v[i] = fmaf(w[i], RESID_SCALE_INV, v[i]);
                        tmem_st32(tb + (uint32_t)(c * 32), v);
                    }
                    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
                }
                asm volatile("tcgen05.fence::before_thread_sync;");
                __syncwarp();
                if (lane == 0) {
                    if (PAIR && rank != 0) {
                        mbar_arrive_remote(cluster_addr(smem_u32(corr_free), 0u));
                        if (REGS) mbar_arrive_remote(cluster_addr(smem_u32(&acc_empty[buf]), 0u));
                    } else {
                        mbar_arrive(corr_free);
                        if (REGS) mbar_arrive(&acc_empty[buf]);
                    }
                }
            }
            const GemmPiece pc = piece_of<GROUPED>(tile, pieces, n_pieces, single);
            int m0, n0, c0;
            piece_tile<BN_, CM_>(pc, tile, rank, m0, n0, c0);
            const int64_t r = (int64_t)m0 + quad * 32 + lane;    // row within the piece
            const int64_t rows = pc.rows, n = pc.n;
            const bool live = r < rows;
            if constexpr (EMIT) {
                // the fused selection: every value of a live row whose order key
                // reaches the row's threshold (tk, read above; dead rows never
                // reach it) is appended to the row's candidate buffer.  Per
                // 32-column chunk a branch-free compare gives the row's hit mask;
                // a row with hits stages the chunk's values in its part of the
                // warp's staging block and copies each hit's word, found by its
                // bit, into its EMIT_SLOTS slots.  The accumulator is released
                // before the row's places are reserved (one atomic per row and
                // tile) and the slots written out; a row with more hits than
                // slots reserves first and writes them during a second pass over
                // its chunks.  Entries past the capacity are dropped (the count
                // still tells).
                constexpr int SLOTS = C::EMIT_SLOTS;
                const int64_t grow = pc.q_row0 + r;
                uint64_t *dst = emit.cand + grow * (int64_t)emit.cap;
                uint64_t *slotw = emit_slots + ((warp - 2) * 32 + lane) * SLOTS;
                float *vst = staging + (warp - 2) * 32 * 32 + lane * 32;   // 32 floats, 16-byte slots swizzled
                const float sr = (MODE == kSimFp8 && live) ? scale_q[pc.q_row0 + r] : 1.f;
                // the row's values of the warp's column chunk cc (32 objects from
                // n0 + 32 (cbase + cc))
                auto chunk = [&](int cc, float (&v)[32]) {
                    if constexpr (REGS) {
#pragma unroll
                        for (int i = 0; i < 32; ++i) v[i] = fv[cc][i];
                        return;
                    }
                    const int c = cbase + cc;
                    const uint32_t lane_addr = tmem + buf * (uint32_t)C::ACC_COLS + ((uint32_t)(quad * 32) << 16) +
                                               (uint32_t)(c * 32);
                    tmem_ld32(lane_addr, v);
                    if (MODE == kSimF16x3 && !FOLD) {
                        float w[32];
                        tmem_ld32(lane_addr + ACC_CORR, w);
#pragma unroll
                        for (int i = 0; i < 32; ++i) v[i] = fmaf(w[i], RESID_SCALE_INV, v[i]);
                    }
                    if (MODE == kSimFp8 && live) {
                        const int64_t obj0 = (int64_t)n0 + c * 32;
                        const float *__restrict__ scale_d = pc.scale_d;
#pragma unroll
                        for (int i = 0; i < 32; ++i)
                            v[i] *= sr * (obj0 + i < n ? __ldg(scale_d + obj0 + i) : 0.f);
                    }
                };
                // the threshold as a float: for non-NaN values v >= tf exactly when
                // order_key(v) >= tk (-0 and +0 compare equal and share a key)
                const bool dead = tk == 0xffffffffu;
                const bool all_pass = tk == 0u;     // a sample shorter than the list: every entry
                const float tf = (dead || all_pass) ? 0.f : key_value(tk);
                uint32_t masks[NCH];
                int nh = 0;
#pragma unroll
                for (int cc = 0; cc < NCH; ++cc) {
                    const int c = cbase + cc;
                    float v[32];
                    chunk(cc, v);
                    const int64_t obj0 = (int64_t)n0 + c * 32;
                    uint32_t hit = 0u;
#pragma unroll
                    for (int i = 0; i < 32; ++i) hit |= (v[i] >= tf || all_pass) ? (1u << i) : 0u;
                    if (obj0 + 32 > n) hit &= obj0 >= n ? 0u : (0xffffffffu >> (32 - (int)(n - obj0)));
                    if (dead) hit = 0u;
                    masks[cc] = hit;
                    if (hit) {
#pragma unroll
                        for (int j = 0; j < 8; ++j)
                            reinterpret_cast<float4 *>(vst)[j ^ (lane & 7)] =
                                make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
                        uint32_t h = hit;
                        while (h) {
                            const int i = __ffs(h) - 1;
                            h &= h - 1u;
                            if (nh < SLOTS) {
                                const float x = vst[(((i >> 2) ^ (lane & 7)) << 2) | (i & 3)];
                                slotw[nh] = ((uint64_t)order_key(x) << 32) |
                                            (uint64_t)(0xffffffffu - (uint32_t)(obj0 + i));
                            }
                            ++nh;
                        }
                    }
                }
                const bool over = nh > SLOTS;
                if (__any_sync(0xffffffffu, over)) {
                    int pos = over ? atomicAdd(emit.cnt + grow, nh) : 0;
#pragma unroll
                    for (int cc = 0; cc < NCH; ++cc) {
                        const int c = cbase + cc;
                        if (!__any_sync(0xffffffffu, over && masks[cc] != 0u)) continue;    // tcgen05.ld is warp-wide
                        float v[32];
                        chunk(cc, v);
                        if (!over) continue;
                        const int64_t obj0 = (int64_t)n0 + c * 32;
#pragma unroll
                        for (int i = 0; i < 32; ++i) {
                            if ((masks[cc] >> i) & 1u) {
                                if (pos < emit.cap)
                                    dst[pos] = ((uint64_t)order_key(v[i]) << 32) |
                                               (uint64_t)(0xffffffffu - (uint32_t)(obj0 + i));
                                ++pos;
                            }
                        }
                    }
                }
                if constexpr (!REGS) {
                    asm volatile("tcgen05.fence::before_thread_sync;");
                    __syncwarp();
                    if (lane == 0) {
                        if (PAIR && rank != 0) mbar_arrive_remote(cluster_addr(smem_u32(&acc_empty[buf]), 0u));
                        else mbar_arrive(&acc_empty[buf]);
                    }
                }
                if (nh > 0 && !over) {
                    const int pos = atomicAdd(emit.cnt + grow, nh);
                    for (int k = 0; k < nh; ++k)
                        if (pos + k < emit.cap) dst[pos + k] = slotw[k];
                }
                continue;
            }
            const int64_t ns_ = pc.n_store;       // valid stored columns (sample tiles compacted)
            const int64_t r_blk = (int64_t)m0 + quad * 32;       // first row of the warp's blocks
            const bool store = pc.s_off >= 0;     // s_off -1: the group maxima only (uniform across the warp)
            float *sblk = S + (store ? pc.s_off : 0) + r_blk * pc.ld;
            const bool vec = (pc.ld % 4) == 0;
            // stored columns c0 + ... are valid below ns_ exactly where their objects n0 + ... are below n
            const float sr = (MODE == kSimFp8 && live) ? scale_q[pc.q_row0 + r] : 1.f;
            // FP8 mode: the tile's column scales (zero past the row end), staged once
            // per tile in the warp's slot instead of one bounds-checked load per entry
            float *scl = tile_scales + (warp - 2) * BN;
            if (MODE == kSimFp8) {
                const float *__restrict__ scale_d = pc.scale_d;
                for (int j = lane; j < BN; j += 32) scl[j] = (int64_t)n0 + j < n ? __ldg(scale_d + n0 + j) : 0.f;
                __syncwarp();
            }
            const bool keep_tops = tops != nullptr && pc.tops_off >= 0;    // uniform across the warp
            float gmax[NCH * 4];     // maximum of each 8-column group of row r in the warp's columns
#pragma unroll
            for (int cc = 0; cc < NCH; ++cc) {
                const int c = cbase + cc;
                float v[32];
                if constexpr (REGS) {
#pragma unroll
                    for (int i = 0; i < 32; ++i) v[i] = fv[cc][i];
                } else {
                    const uint32_t lane_addr = tmem + buf * (uint32_t)C::ACC_COLS + ((uint32_t)(quad * 32) << 16) +
                                               (uint32_t)(c * 32);
                    tmem_ld32(lane_addr, v);
                    if (MODE == kSimF16x3 && !FOLD) {
                        float w[32];
                        tmem_ld32(lane_addr + ACC_CORR, w);
#pragma unroll
                        for (int i = 0; i < 32; ++i) v[i] = fmaf(w[i], RESID_SCALE_INV, v[i]);
                    }
                }
                const int64_t col0 = (int64_t)c0 + c * 32;      // stored column
                if (MODE == kSimFp8 && live) {
                    const float4 *s4 = reinterpret_cast<const float4 *>(scl + c * 32);
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        const float4 t = s4[q];
                        v[4 * q] *= sr * t.x;
                        v[4 * q + 1] *= sr * t.y;
                        v[4 * q + 2] *= sr * t.z;
                        v[4 * q + 3] *= sr * t.w;
                    }
                }
                if (keep_tops) {
                    const float ninf = -__int_as_float(0x7f800000);
#pragma unroll
                    for (int g = 0; g < 4; ++g) {
                        float m = ninf;
                        if (col0 + 32 <= ns_) {
#pragma unroll
                            for (int i = 0; i < 8; ++i) m = fmaxf(m, v[8 * g + i]);
                        } else {
#pragma unroll
                            for (int i = 0; i < 8; ++i)
                                if (col0 + 8 * g + i < ns_) m = fmaxf(m, v[8 * g + i]);
                        }
                        gmax[4 * cc + g] = m;
                    }
                }
                if (!store) continue;
#pragma unroll
                for (int j = 0; j < 8; ++j)
                    blk[lane * 8 + (j ^ (lane & 7))] = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
                __syncwarp();
                const int64_t cs = col0 + slot * 4;
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const int rr = 4 * i + sub;
                    const float4 x = blk[rr * 8 + (slot ^ (rr & 7))];
                    if (r_blk + rr < rows) {
                        float *dst = sblk + (int64_t)rr * pc.ld + cs;
                        if (vec && cs + 4 <= ns_) {
                            *reinterpret_cast<float4 *>(dst) = x;
                        } else {
                            if (cs < ns_) dst[0] = x.x;
                            if (cs + 1 < ns_) dst[1] = x.y;
                            if (cs + 2 < ns_) dst[2] = x.z;
                            if (cs + 3 < ns_) dst[3] = x.w;
                        }
                    }
                }
                __syncwarp();
            }
            if (keep_tops) {
                const int64_t gs = group_stride(ns_, pc.gshift);
                float *tblk = tops + pc.tops_off + r_blk * gs;
                // (the warp's groups start at group c0 / 8 + 4 cbase, of 32: c0 / 32 + cbase)
                if (pc.gshift == kGroupShiftSmall) {
                    float4 t4[NCH];
#pragma unroll
                    for (int j = 0; j < NCH; ++j)
                        t4[j] = make_float4(gmax[4 * j], gmax[4 * j + 1], gmax[4 * j + 2], gmax[4 * j + 3]);
                    store_rows_staged<NCH>(blk, t4, lane, tblk + c0 / 8 + 4 * cbase, gs, rows - r_blk);
                } else {
                    float4 t4[NCH / 4];
#pragma unroll
                    for (int j = 0; j < NCH / 4; ++j) {
                        float g4[4];
#pragma unroll
                        for (int u = 0; u < 4; ++u)
                            g4[u] = fmaxf(fmaxf(gmax[16 * j + 4 * u], gmax[16 * j + 4 * u + 1]),
                                          fmaxf(gmax[16 * j + 4 * u + 2], gmax[16 * j + 4 * u + 3]));
                        t4[j] = make_float4(g4[0], g4[1], g4[2], g4[3]);
                    }
                    store_rows_staged<NCH / 4>(blk, t4, lane, tblk + c0 / 32 + cbase, gs, rows - r_blk);
                }
            }
            if constexpr (!REGS) {
                asm volatile("tcgen05.fence::before_thread_sync;");
                __syncwarp();
                if (lane == 0) {
                    if (PAIR && rank != 0) mbar_arrive_remote(cluster_addr(smem_u32(&acc_empty[buf]), 0u));
                    else mbar_arrive(&acc_empty[buf]);
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncwarp();      // warps 0 and 1 ran their roles on lane 0 only
    cluster_sync();    // no CTA leaves while a peer's copies or commits may still target its shared memory
    if (warp == 1) {
        asm volatile("tcgen05.fence::after_thread_sync;");
        if (PAIR) asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_ALLOC));
        else asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_ALLOC));
    }
}

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;

bool get_encoder()
{
    if (g_encode) return true;
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn)
        return false;
    g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    return true;
}

// 2D tensor [outer, inner] row-major (FP16, BF16 or FP8 bytes), box
// [box_outer, BK], swizzle matching the mode's row width.
template <int MODE>
bool make_map(CUtensorMap *m, const void *base, int64_t inner, int64_t outer, int box_outer)
{
    using M = Elem<MODE>;
    const int esize = MODE == kSimFp8 ? 1 : 2;
    const CUtensorMapDataType dt = MODE == kSimF16x3 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                   : (MODE == kSimBf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_UINT8);
    cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)outer};
    cuuint64_t strides[1] = {(cuuint64_t)inner * esize};
    cuuint32_t box[2] = {(cuuint32_t)M::BK, (cuuint32_t)box_outer};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = g_encode(m, dt, 2, const_cast<void *>(base), dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE,
                          MODE == kSimF16x3 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_128B,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

// Launch with the cluster attribute and a persistent grid of as many clusters
// as can be resident at once (a GPC with an odd number of free SMs cannot
// hold a whole cluster on its last SM); the count is cached per device and
// kernel (concurrent first calls compute the same value).
template <int MODE, int BN_, int CM_, bool GROUPED, bool PAIR = false, bool EMIT = false>
cudaError_t launch_impl(const CUtensorMap &mq0, const CUtensorMap &mq1, const CUtensorMap &md0,
                        const CUtensorMap &md1, const GemmPiece *pieces, int32_t n_pieces, const GemmPiece &single,
                        float *S, float *tops, int32_t k_slices, int64_t total_tiles, const float *scale_q,
                        int num_sms, int32_t *err, cudaStream_t s, const FuseEmit &emit = FuseEmit{})
{
    using C = Cfg<MODE, BN_, CM_, PAIR, EMIT>;
    if (total_tiles <= 0) return cudaSuccess;
    if (total_tiles > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    auto kernel = sim_tc_kernel<MODE, BN_, CM_, GROUPED, PAIR, EMIT>;
    const int smem_bytes = C::SMEM_BYTES;
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.blockDim = dim3(C::THREADS);
    cfg.dynamicSmemBytes = smem_bytes;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CM_;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    static int resident[64] = {};      // per device, per kernel instantiation
    int dev = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    int *slot = dev >= 0 && dev < 64 ? &resident[dev] : nullptr;
    int nc = slot ? *slot : 0;
    if (nc == 0) {
        cfg.gridDim = dim3((unsigned)(std::max(num_sms / CM_, 1) * CM_));
        if (cudaOccupancyMaxActiveClusters(&nc, kernel, &cfg) != cudaSuccess || nc < 1) {
            (void)cudaGetLastError();    // the query's error is not the launch's
            nc = std::max(num_sms / CM_, 1);
        }
        if (slot) *slot = nc;
    }
    const int clusters = (int)std::min<int64_t>(total_tiles, nc);
    cfg.gridDim = dim3((unsigned)(clusters * CM_));
    e = cudaLaunchKernelEx(&cfg, kernel, mq0, mq1, md0, md1, pieces, n_pieces, single, S, tops, k_slices,
                           (int32_t)total_tiles, scale_q, err, emit);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

// Rows are padded to kDimAlign (64) elements; the FP8 K slice (128 bytes) may
// run past the row end, where the tensor map's bounds fill zeros.
template <int MODE>
int32_t k_slices_of(int32_t dim_pad)
{
    return (dim_pad + Elem<MODE>::BK - 1) / Elem<MODE>::BK;
}

// One problem, tile configuration 2 (256 x 256 tiles on CTA pairs).
template <int MODE>
cudaError_t launch_tc(const void *q0, const void *q1, const void *d0, const void *d1, float *S, int64_t rows,
                      int64_t n, int32_t dim_pad, int64_t ld_s, const float *scale_q, const float *scale_d,
                      float *tops, int num_sms, int32_t *err, cudaStream_t s)
{
    constexpr int BN_ = 256, CM_ = 2;
    static_assert(BN_ == 256 && CM_ == 2, "the tile count below is that of the pair variant");
    constexpr bool TWO = !Elem<MODE>::SPLIT;
    if (rows <= 0 || n <= 0) return cudaSuccess;
    if (sim_variant_bn(kSimPairVariant) != BN_ || sim_variant_cluster(kSimPairVariant) != CM_)
        return cudaErrorInvalidConfiguration;
    if (dim_pad % kDimAlign != 0 || rows > 0x7fffffffLL || n > 0x7fffffffLL || ld_s < n || ld_s > 0x7fffffffLL)
        return cudaErrorInvalidValue;
    if (!get_encoder()) return cudaErrorNotSupported;
    // TMA: 16-byte aligned bases; row strides are multiples of 16 bytes (dim_pad % 64 == 0)
    const uintptr_t al = (uintptr_t)q0 | (uintptr_t)d0 | (TWO ? 0 : ((uintptr_t)q1 | (uintptr_t)d1));
    if (al & 15u) return cudaErrorMisalignedAddress;
    if (tops && ((uintptr_t)tops & 15u)) return cudaErrorMisalignedAddress;
    if (MODE == kSimFp8 && (!scale_q || !scale_d)) return cudaErrorInvalidValue;
    CUtensorMap mq0, mq1, md0, md1;
    if (!make_map<MODE>(&mq0, q0, dim_pad, rows, BM) || !make_map<MODE>(&md0, d0, dim_pad, n, BN_ / CM_))
        return cudaErrorInvalidValue;
    if (TWO) {
        mq1 = mq0;
        md1 = md0;
    } else if (!make_map<MODE>(&mq1, q1, dim_pad, rows, BM) || !make_map<MODE>(&md1, d1, dim_pad, n, BN_ / CM_)) {
        return cudaErrorInvalidValue;
    }
    GemmPiece single{};
    single.q_row0 = 0;
    single.s_off = 0;
    single.tops_off = tops ? 0 : -1;
    single.scale_d = scale_d;
    single.bmap = nullptr;
    single.rows = (int32_t)rows;
    single.n = (int32_t)n;
    single.ld = (int32_t)ld_s;
    single.tile_begin = 0;
    single.gshift = group_shift_for(n);
    single.col_mode = kColAll;
    single.col_stride = 0;
    single.n_store = (int32_t)n;
    return launch_impl<MODE, BN_, CM_, false, true>(mq0, mq1, md0, md1, nullptr, 1, single, S, tops,
                                              k_slices_of<MODE>(dim_pad), sim_cluster_tiles(rows, n, kSimPairVariant), scale_q,
                                              num_sms, err, s);
}

template <int MODE, int BN_, int CM_, bool PAIR = false>
cudaError_t launch_grouped(const void *q0, const void *q1, int64_t rows_total, int32_t dim_pad,
                           const GemmPiece *pieces, int32_t n_pieces, int64_t total_tiles, float *S, float *tops,
                           const float *scale_q, int num_sms, int32_t *err, cudaStream_t s, const FuseEmit *emit)
{
    constexpr bool TWO = !Elem<MODE>::SPLIT;
    if (total_tiles <= 0) return cudaSuccess;
    if (n_pieces < 1 || rows_total < 1 || rows_total > 0x7fffffffLL || dim_pad % kDimAlign != 0 || !pieces)
        return cudaErrorInvalidValue;
    if (!get_encoder()) return cudaErrorNotSupported;
    const uintptr_t al = (uintptr_t)q0 | (TWO ? 0 : (uintptr_t)q1) | (uintptr_t)S | (tops ? (uintptr_t)tops : 0);
    if (al & 15u) return cudaErrorMisalignedAddress;
    if (MODE == kSimFp8 && !scale_q) return cudaErrorInvalidValue;
    CUtensorMap mq0, mq1;
    if (!make_map<MODE>(&mq0, q0, dim_pad, rows_total, BM)) return cudaErrorInvalidValue;
    if (TWO) mq1 = mq0;
    else if (!make_map<MODE>(&mq1, q1, dim_pad, rows_total, BM)) return cudaErrorInvalidValue;
    GemmPiece unused{};
    // the B maps of the pieces live in device memory; map_d0 / map_d1 are unused
    if (emit) {
        if constexpr (BN_ == 256) {
            if (!emit->tau_key || !emit->cnt || !emit->cand || emit->cap < 1) return cudaErrorInvalidValue;
            return launch_impl<MODE, BN_, CM_, true, PAIR, true>(mq0, mq1, mq0, mq1, pieces, n_pieces, unused, S,
                                                           tops, k_slices_of<MODE>(dim_pad), total_tiles, scale_q,
                                                           num_sms, err, s, *emit);
        }
        return cudaErrorInvalidValue;     // the fused selection samples tiles of 256 objects
    }
    return launch_impl<MODE, BN_, CM_, true, PAIR>(mq0, mq1, mq0, mq1, pieces, n_pieces, unused, S, tops,
                                             k_slices_of<MODE>(dim_pad), total_tiles, scale_q, num_sms, err, s);
}

template <int MODE>
cudaError_t launch_grouped_variant(int variant, const void *q0, const void *q1, int64_t rows_total, int32_t dim_pad,
                                   const GemmPiece *pieces, int32_t n_pieces, int64_t total_tiles, float *S,
                                   float *tops, const float *scale_q, int num_sms, int32_t *err, cudaStream_t s,
                                   const FuseEmit *emit)
{
    switch (variant) {
    case 0:
        return launch_grouped<MODE, 256, 1>(q0, q1, rows_total, dim_pad, pieces, n_pieces, total_tiles, S, tops,
                                            scale_q, num_sms, err, s, emit);
    case 1:
        return launch_grouped<MODE, 128, 1>(q0, q1, rows_total, dim_pad, pieces, n_pieces, total_tiles, S, tops,
                                            scale_q, num_sms, err, s, emit);
    case 2:
        return launch_grouped<MODE, 256, 2, true>(q0, q1, rows_total, dim_pad, pieces, n_pieces, total_tiles, S,
                                                  tops, scale_q, num_sms, err, s, emit);
    default:
        return cudaErrorInvalidValue;
    }
}

template <int MODE>
bool encode_b_variant(void *out, const void *d0, const void *d1, int64_t n, int32_t dim_pad, int variant)
{
    CUtensorMap *m = static_cast<CUtensorMap *>(out);
    const int box = sim_variant_bn(variant) / sim_variant_cluster(variant);
    return make_map<MODE>(&m[0], d0, dim_pad, n, box) && make_map<MODE>(&m[1], d1 ? d1 : d0, dim_pad, n, box);
}

}  // namespace

bool sim_tc_available() { return get_encoder(); }

bool sim_tc_encode_b(int mode, int variant, void *out, const void *d0, const void *d1, int64_t n, int32_t dim_pad)
{
    static_assert(sizeof(CUtensorMap) == kTensorMapBytes, "tensor map size");
    if (!get_encoder() || n < 1 || variant < 0 || variant >= kSimVariants || (reinterpret_cast<uintptr_t>(out) & 63u))
        return false;
    switch (mode) {
    case kSimF16x3: return encode_b_variant<kSimF16x3>(out, d0, d1, n, dim_pad, variant);
    case kSimBf16: return encode_b_variant<kSimBf16>(out, d0, nullptr, n, dim_pad, variant);
    case kSimFp8: return encode_b_variant<kSimFp8>(out, d0, nullptr, n, dim_pad, variant);
    default: return false;
    }
}

cudaError_t launch_sim_tc_grouped(int mode, int variant, const void *q0, const void *q1, int64_t rows_total,
                                  int32_t dim_pad, const GemmPiece *pieces, int32_t n_pieces, int64_t total_tiles,
                                  float *S, float *tops, const float *scale_q, int num_sms, int32_t *err,
                                  cudaStream_t s, const FuseEmit *emit)
{
    switch (mode) {
    case kSimF16x3:
        return launch_grouped_variant<kSimF16x3>(variant, q0, q1, rows_total, dim_pad, pieces, n_pieces, total_tiles,
                                                 S, tops, scale_q, num_sms, err, s, emit);
    case kSimBf16:
        return launch_grouped_variant<kSimBf16>(variant, q0, q1, rows_total, dim_pad, pieces, n_pieces, total_tiles,
                                                S, tops, scale_q, num_sms, err, s, emit);
    case kSimFp8:
        return launch_grouped_variant<kSimFp8>(variant, q0, q1, rows_total, dim_pad, pieces, n_pieces, total_tiles,
                                               S, tops, scale_q, num_sms, err, s, emit);
    default:
        return cudaErrorInvalidValue;
    }
}

cudaError_t launch_sim_tc_f16x3(const uint16_t *q_hi, const uint16_t *q_lo, const uint16_t *d_hi,
                                const uint16_t *d_lo, float *S, int64_t rows, int64_t n, int32_t dim_pad, int64_t ld_s,
                                float *tops, int num_sms, int32_t *err, cudaStream_t s)
{
    return launch_tc<kSimF16x3>(q_hi, q_lo, d_hi, d_lo, S, rows, n, dim_pad, ld_s, nullptr, nullptr, tops, num_sms,
                                err, s);
}

cudaError_t launch_sim_tc_bf16(const uint16_t *q, const uint16_t *d, float *S, int64_t rows, int64_t n,
                               int32_t dim_pad, int64_t ld_s, float *tops, int num_sms, int32_t *err, cudaStream_t s)
{
    return launch_tc<kSimBf16>(q, nullptr, d, nullptr, S, rows, n, dim_pad, ld_s, nullptr, nullptr, tops, num_sms,
                               err, s);
}

cudaError_t launch_sim_tc_fp8(const uint8_t *q, const float *scale_q, const uint8_t *d, const float *scale_d,
                              float *S, int64_t rows, int64_t n, int32_t dim_pad, int64_t ld_s, float *tops,
                              int num_sms, int32_t *err, cudaStream_t s)
{
    return launch_tc<kSimFp8>(q, nullptr, d, nullptr, S, rows, n, dim_pad, ld_s, scale_q, scale_d, tops, num_sms,
                              err, s);
}

// Loads the single-problem FP32-accurate kernel (CTA pairs; modules and
// functions load lazily on first use).
cudaError_t preload_sim_tc_f16x3()
{
    cudaFuncAttributes a;
    return cudaFuncGetAttributes(&a, sim_tc_kernel<kSimF16x3, 256, 2, false, true>);
}

}  // namespace farm
