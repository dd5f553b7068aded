// k_fuse.cu -- reciprocal-rank fusion of several retrieval channels
// (App. D.2 step 3): the target similarity of an object is
//   F(j) = sum_c w_c / (mu + rank_c(j))
// over the query's channels, s_sem = cf * F, and landmark variables are
// retrieved the same way (L_i = the K_a objects of largest fused score).
//
// Input per row (a target row of a query, or a landmark row of a
// constraint): every channel's list of its R best objects in rank order (the
// rank select over that channel's similarity row) and the channel's whole
// similarity row.  One CTA per row:
//  1. the union of the channels' lists (a shared-memory hash on the object
//     index), with each member's rank in the channels that list it;
//  2. bounds on every member's F: a channel that did not list it ranks it in
//     [R + 1, n], so F lies in [LB, UB] (computed with the same operations
//     and order as F itself, hence bracketing it in FP32 too);
//  3. the members that can still matter: for a target row those with
//     cf * UB >= (1 - w) * (k_max-th largest cf * LB) -- the composite of
//     App. D.2 step 5 is at least (1 - w) s_sem, so the others cannot reach
//     the TopK -- or UB >= the k_closest-th largest LB (the Closest /
//     Farthest candidate set); for a landmark row those with UB >= the K_a-th
//     largest LB;
//  4. their exact rank in each channel that did not list them, by counting
//     the row's entries above them: rank = 1 + #{j : c_j > c_e, or equal and
//     j < e} (the probes sorted once, each entry of the row placed among them
//     by binary search; groups whose maximum -- from the similarity epilogue
//     -- is below the smallest probe are skipped);
//  5. exact F in FP32, and the kept members sorted by (F desc, index asc):
//     a target row writes them (and their count to the query's metadata) for
//     the compose kernel, a landmark row writes its first K_a.
// Objects outside every list score F <= W / (mu + R + 1); the host picks R
// so that this stays below the thresholds of step 3.
#include "select_common.cuh"

namespace farm {
namespace {

using namespace sel;

constexpr int TF = 256;

// Dynamic shared memory of one row, sized by the launch's largest entry count
// E (channels x list length), P2 = the power of two >= E and the hash size
// H (a power of two >= 1.5 E).  Region A holds the hash while the union is
// built, then the probes with their histogram, then the output sort (over
// the probes' words); region B holds the members.
struct FuseSmem {
    size_t hkey, hrank, probe, pslot, phist, skey;   // region A
    size_t midx, mrank, lb, ub, k32, surv;           // region B
    size_t bytes;
    __host__ __device__ static size_t up16(size_t x) { return (x + 15) & ~(size_t)15; }
    __host__ __device__ FuseSmem(int E, int H, int P2)
    {
        size_t a = 0;
        hkey = a;  a = up16(a + (size_t)H * 4);
        hrank = a; a = up16(a + (size_t)H * FARM_MAX_CHANNELS * 2);
        const size_t a_hash = a;
        a = 0;
        probe = a; a = up16(a + (size_t)P2 * 8);
        skey = probe;                                // (the output sort follows the last probe pass)
        pslot = a; a = up16(a + (size_t)P2 * 4);
        phist = a; a = up16(a + (size_t)(E + 1) * 4);
        const size_t a_end = a_hash > a ? a_hash : a;
        size_t b = a_end;
        midx = b;  b = up16(b + (size_t)E * 4);
        mrank = b; b = up16(b + (size_t)E * FARM_MAX_CHANNELS * 4);
        lb = b;    b = up16(b + (size_t)E * 4);
        ub = b;    b = up16(b + (size_t)E * 4);
        k32 = b;   b = up16(b + (size_t)E * 4);
        surv = b;  b = up16(b + (size_t)E * 4);
        bytes = b;
    }
    __host__ __device__ static int hash_size(int E)
    {
        int H = 1;
        while (H < E + (E >> 1) + 1) H <<= 1;
        return H;
    }
    __host__ __device__ static int pow2(int E)
    {
        int P = 1;
        while (P < E) P <<= 1;
        return P;
    }
};

__device__ __forceinline__ uint64_t entry_key(float v, int32_t j)
{
    return ((uint64_t)order_key(v) << 32) | (uint64_t)(0xffffffffu - (uint32_t)j);
}

// Fused score with the channels' ranks (0: unlisted, counted as rank `miss`).
__device__ __forceinline__ float fused(const FuseArgs &a, const int32_t *rk, float miss)
{
    float f = 0.f;
    for (int c = 0; c < a.n_ch; ++c) f += a.w[c] / (a.p.mu + (rk[c] > 0 ? (float)rk[c] : miss));
    return f;
}

__global__ void __launch_bounds__(TF)
fuse_kernel(FuseArgs a, int64_t b0, int32_t E, int32_t H, int32_t P2)
{
    extern __shared__ __align__(16) uint8_t sm[];
    const FuseSmem L(E, H, P2);
    int32_t *hkey = reinterpret_cast<int32_t *>(sm + L.hkey);
    uint16_t *hrank = reinterpret_cast<uint16_t *>(sm + L.hrank);
    uint64_t *probe = reinterpret_cast<uint64_t *>(sm + L.probe);
    int32_t *pslot = reinterpret_cast<int32_t *>(sm + L.pslot);
    uint32_t *phist = reinterpret_cast<uint32_t *>(sm + L.phist);
    uint64_t *skey = reinterpret_cast<uint64_t *>(sm + L.skey);
    int32_t *midx = reinterpret_cast<int32_t *>(sm + L.midx);
    int32_t *mrank = reinterpret_cast<int32_t *>(sm + L.mrank);
    float *lb = reinterpret_cast<float *>(sm + L.lb);
    float *ub = reinterpret_cast<float *>(sm + L.ub);
    uint32_t *k32 = reinterpret_cast<uint32_t *>(sm + L.k32);
    int32_t *surv = reinterpret_cast<int32_t *>(sm + L.surv);
    __shared__ uint32_t hist[2048];
    __shared__ uint32_t wsum[TF / 32];
    __shared__ uint32_t s3[3];
    __shared__ int s_u, s_ns, s_np;
    __shared__ float s_thr[2];

    const int tid = threadIdx.x;
    const int64_t b = b0 + blockIdx.x;      // rows: targets 0 .. n_q-1, then landmarks
    const bool tgt = b < a.n_q;
    const int64_t row = b;                                  // row of every channel's similarity block
    const int R = tgt ? a.Rt : a.Rl;                        // list length of every channel
    const int32_t *lists = tgt ? a.tlist : a.llist;
    const int64_t lrow = tgt ? b : b - a.n_q;
    const int64_t lrows = tgt ? a.n_q : a.n_c;
    const int n = a.n;
    const int nch = a.n_ch;
    int c_t = -1;
    if (tgt) c_t = a.qmeta[b * 8 + QM_CLS];

    // 1. union of the channels' lists
    for (int s = tid; s < H; s += TF) {
        hkey[s] = -1;
        for (int c = 0; c < FARM_MAX_CHANNELS; ++c) hrank[s * FARM_MAX_CHANNELS + c] = 0;
    }
    if (tid == 0) { s_u = 0; s_ns = 0; }
    __syncthreads();
    const int hbits = 31 - __clz(H);
    for (int t = tid; t < nch * R; t += TF) {
        const int c = t / R, pos = t - c * R;
        const int32_t e = lists[((int64_t)c * lrows + lrow) * R + pos];
        if (e < 0 || e >= n) continue;
        uint32_t s = ((uint32_t)e * 2654435761u) >> (32 - hbits);
        // the table holds at most E < H keys, so an empty or matching slot is always found
        for (int probe_n = 0; probe_n < H; ++probe_n) {
            const int32_t old = atomicCAS(&hkey[s], -1, e);
            if (old == -1 || old == e) {
                hrank[s * FARM_MAX_CHANNELS + c] = (uint16_t)(pos + 1);
                break;
            }
            s = (s + 1) & (uint32_t)(H - 1);
        }
    }
    __syncthreads();
    for (int s = tid; s < H; s += TF) {
        if (hkey[s] >= 0) {
            const int m = atomicAdd(&s_u, 1);
            midx[m] = hkey[s];
            for (int c = 0; c < FARM_MAX_CHANNELS; ++c) mrank[m * FARM_MAX_CHANNELS + c] = hrank[s * FARM_MAX_CHANNELS + c];
        }
    }
    __syncthreads();
    const int U = s_u;

    // 2. bounds (a channel that did not list a member ranks it in [R + 1, n])
    const bool complete = R >= n;     // every list holds every object
    for (int m = tid; m < U; m += TF) {
        const int32_t *rk = mrank + m * FARM_MAX_CHANNELS;
        const float cf = (tgt && c_t >= 0 && a.cls[midx[m]] != c_t) ? a.p.class_mis : 1.f;
        const float lo = fused(a, rk, (float)n), hi = complete ? lo : fused(a, rk, (float)(R + 1));
        lb[m] = lo;
        ub[m] = hi;
        k32[m] = order_key(cf * lo);
    }
    __syncthreads();

    // 3. thresholds: the K-th largest lower bound
    if (tid == 0) { s_thr[0] = -__int_as_float(0x7f800000); s_thr[1] = -__int_as_float(0x7f800000); }
    __syncthreads();
    const int K0 = tgt ? a.p.k_max : a.p.k_anchor;
    if (K0 <= U) {
        const float v = key_value(kth_key<TF>(k32, U, K0, hist, wsum, s3));
        if (tid == 0) s_thr[0] = tgt ? (1.f - a.p.w) * v : v;
    }
    __syncthreads();
    if (tgt) {
        for (int m = tid; m < U; m += TF) k32[m] = order_key(lb[m]);
        __syncthreads();
        const int kc = min(a.p.k_closest, n);
        if (kc <= U) {
            const float v = key_value(kth_key<TF>(k32, U, kc, hist, wsum, s3));
            if (tid == 0) s_thr[1] = v;
        }
        __syncthreads();
    }
    const float thr0 = s_thr[0], thr1 = s_thr[1];
    for (int m = tid; m < U; m += TF) {
        const float cf = (tgt && c_t >= 0 && a.cls[midx[m]] != c_t) ? a.p.class_mis : 1.f;
        const bool keep = tgt ? (cf * ub[m] >= thr0 || ub[m] >= thr1) : ub[m] >= thr0;
        if (keep) surv[atomicAdd(&s_ns, 1)] = m;
    }
    __syncthreads();
    const int ns = s_ns;

    // 4. exact ranks of the kept members in the channels that did not list them
    if (!complete) {
        for (int c = 0; c < nch; ++c) {
            const float *srow = a.S + ((int64_t)c * a.rows + row) * a.ld;
            if (tid == 0) s_np = 0;
            __syncthreads();
            for (int k = tid; k < ns; k += TF) {
                const int m = surv[k];
                if (mrank[m * FARM_MAX_CHANNELS + c] == 0) {
                    const int i = atomicAdd(&s_np, 1);
                    probe[i] = entry_key(srow[midx[m]], midx[m]);
                    pslot[i] = m;
                }
            }
            __syncthreads();
            const int np = s_np;
            if (np == 0) continue;        // (uniform: every thread read s_np after the barrier)
            int P = 1;
            while (P < np) P <<= 1;
            for (int i = np + tid; i < P; i += TF) { probe[i] = ~0ull; pslot[i] = -1; }
            for (int i = tid; i <= np; i += TF) phist[i] = 0;
            __syncthreads();
            // ascending bitonic sort of the probes with their member slots
            for (int k = 2; k <= P; k <<= 1) {
                for (int j = k >> 1; j > 0; j >>= 1) {
                    for (int i = tid; i < P; i += TF) {
                        const int ixj = i ^ j;
                        if (ixj > i) {
                            const uint64_t x = probe[i], y = probe[ixj];
                            const bool up = (i & k) == 0;
                            if (up ? (x > y) : (x < y)) {
                                probe[i] = y; probe[ixj] = x;
                                const int32_t t = pslot[i]; pslot[i] = pslot[ixj]; pslot[ixj] = t;
                            }
                        }
                    }
                    __syncthreads();
                }
            }
            // every entry j beats the probes whose key is below its own; an
            // entry below the smallest probe's value beats none, so groups
            // whose maximum is below it are not read
            const float vmin = key_value((uint32_t)(probe[0] >> 32));
            const float *trow = a.tops + ((int64_t)c * a.rows + row) * a.gstride;
            for (int j = tid; j < n; j += TF) {
                if (trow[j >> a.gshift] < vmin) continue;
                const uint64_t kj = entry_key(__ldcs(srow + j), j);
                int lo = 0, hi = np;          // first probe with key >= kj
                while (lo < hi) {
                    const int mid = (lo + hi) >> 1;
                    if (probe[mid] < kj) lo = mid + 1;
                    else hi = mid;
                }
                if (lo > 0) atomicAdd(&phist[lo], 1u);
            }
            __syncthreads();
            // rank of probe i = 1 + #{entries placed above it} = 1 + sum of phist[i+1 .. np]
            if (tid == 0) {
                uint32_t acc = 0;
                for (int i = np - 1; i >= 0; --i) {
                    acc += phist[i + 1];
                    mrank[pslot[i] * FARM_MAX_CHANNELS + c] = (int32_t)(1 + acc);
                }
            }
            __syncthreads();
        }
    }

    // 5. exact F of the kept members, sorted by (F desc, index asc)
    int P = 1;
    while (P < ns) P <<= 1;
    for (int k = tid; k < P; k += TF) {
        if (k < ns) {
            const int m = surv[k];
            const float f = fused(a, mrank + m * FARM_MAX_CHANNELS, 0.f);
            skey[k] = entry_key(f, midx[m]);
        } else {
            skey[k] = 0ull;
        }
    }
    __syncthreads();
    bitonic_desc<TF>(skey, P);
    if (tgt) {
        const int nout = min(ns, a.RF);
        int32_t *oi = a.out_tidx + b * a.RF;
        float *of = a.out_tF + b * a.RF;
        for (int k = tid; k < a.RF; k += TF) {
            if (k < nout) {
                const int32_t e = (int32_t)(0xffffffffu - (uint32_t)(skey[k] & 0xffffffffu));
                oi[k] = e;
                of[k] = key_value((uint32_t)(skey[k] >> 32));
            } else {
                oi[k] = -1;
                of[k] = 0.f;
            }
        }
        if (tid == 0) {
            a.qmeta[b * 8 + QM_R] = nout;
            if (ns > a.RF) atomicOr(a.err, kErrFusedOverflow);
        }
    } else {
        int32_t *oi = a.out_lidx + lrow * a.Ka;
        for (int k = tid; k < a.Ka; k += TF)
            oi[k] = k < ns ? (int32_t)(0xffffffffu - (uint32_t)(skey[k] & 0xffffffffu)) : -1;
    }
}

}  // namespace

// part 0: the n_q target rows; part 1: the n_c landmark rows (their lists
// are shorter, so their launch needs less shared memory per CTA).
cudaError_t launch_fuse(const FuseArgs &a, int part, cudaStream_t s)
{
    const int64_t blocks = part == 0 ? a.n_q : a.n_c;
    if (blocks <= 0) return cudaSuccess;
    if (a.n_ch < 1 || a.n_ch > FARM_MAX_CHANNELS || a.Rt < 1 || a.Rt > 2 * kMaxTargetCands || a.Rl < 1 ||
        a.Rl > kMaxTargetCands || a.RF < 1 || a.Ka < 1 || a.Ka > a.Rl || a.n_q + a.n_c > 0x7fffffff)
        return cudaErrorInvalidValue;
    const int32_t E = a.n_ch * (part == 0 ? a.Rt : a.Rl);
    const int H = FuseSmem::hash_size(E), P2 = FuseSmem::pow2(E);
    const FuseSmem L(E, H, P2);
    if (L.bytes > 200 * 1024) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(fuse_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.bytes);
    if (e != cudaSuccess) return e;
    fuse_kernel<<<(unsigned)blocks, TF, L.bytes, s>>>(a, part == 0 ? 0 : a.n_q, E, H, P2);
    return cudaGetLastError();
}

}  // namespace farm
