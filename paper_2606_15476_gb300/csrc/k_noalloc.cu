// k_noalloc.cu -- farm_rank_rows_noalloc: ranked object lists for embedding
// rows, computed without any device allocation at call time.
//
// Some callers cannot allocate GPU memory while they serve queries: a process
// on a robot whose GPU memory budget is fixed when it starts (the mapping
// pipeline and model workers own the rest), or a real-time loop that must not
// call cudaMalloc/cudaFree because those calls may synchronise the device and
// take unbounded time.  farm_query_batch grows its workspace on demand, so for
// them this entry point runs the same steps -- normalise the rows, the
// similarity product against a scene's descriptors, the per-row rank select --
// with every intermediate array in one statically allocated device array.
//
// The array is a file-scope __device__ variable.  Host code cannot use the
// variable's name as a device address (on the host it is only a stand-in),
// so farm_create resolves the address with cudaGetSymbolAddress once per
// device, with that device current, and every kernel receives that pointer.
// Resolving the symbol also loads this file's device module (modules load
// lazily), so the array's memory is taken when the first context on the
// device is created, not inside a call of the entry point; the device keeps
// it until the process exits.  The kernels the entry point launches are
// loaded at the same time.
#include <mutex>

#include "farm_internal.h"

namespace farm {
namespace {

// 32 MiB: e.g. 350 rows against a 20,000-object scene at D = 1152.
constexpr size_t kScratchBytes = FARM_NOALLOC_SCRATCH_BYTES;
__device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
void *g_scratch_ptr[kMaxDevices] = {};

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

// Resolves the scratch array's device address for `device` (which must be the
// current device) unless that is done already.  Called by farm_create.
cudaError_t noalloc_setup(int device)
{
    if (device < 0 || device >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (g_scratch_ptr[device]) return cudaSuccess;
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    if (!p) return cudaErrorInvalidSymbol;
    // the kernels of the entry point, loaded now for the same reason
    cudaError_t el = preload_prep();
    if (el == cudaSuccess) el = preload_sim_simt();
    if (el == cudaSuccess) el = preload_select_rows();
    if (el == cudaSuccess && sim_tc_available()) el = preload_sim_tc_f16x3();
    if (el != cudaSuccess) return el;
    g_scratch_ptr[device] = p;
    return cudaSuccess;
}

}  // namespace farm

using farm::Ctx;

extern "C" farm_status farm_rank_rows_noalloc(farm_ctx *ctx, int32_t scene_id, int64_t n_rows, const float *emb,
                                              int32_t r, int32_t precision, int32_t *out_idx, float *out_cos)
{
    if (!ctx) return FARM_EINVAL;
    Ctx &c = *farm::ctx_of(ctx);
    auto fail = [&](farm_status st, const char *msg) {
        c.err = msg;
        return st;
    };
    if (scene_id < 0 || scene_id >= (int32_t)c.scenes.size() || !c.scenes[scene_id].present)
        return fail(FARM_EINVAL, "farm_rank_rows_noalloc: unknown scene");
    if (n_rows < 0) return fail(FARM_EINVAL, "farm_rank_rows_noalloc: n_rows must be >= 0");
    if (n_rows == 0) return FARM_OK;
    if (!emb || !out_idx) return fail(FARM_EINVAL, "farm_rank_rows_noalloc: emb and out_idx must be non-null");
    if (precision != FARM_PREC_FP32 && precision != FARM_PREC_FP32_SIMT)
        return fail(FARM_EINVAL, "farm_rank_rows_noalloc: precision must be FARM_PREC_FP32 or FARM_PREC_FP32_SIMT");
    const farm::Scene &s = c.scenes[scene_id];
    if (r < 1 || r > farm::kMaxTargetCands || r > s.n)
        return fail(FARM_EINVAL, "farm_rank_rows_noalloc: r must lie in [1, min(512, n)]");
    // scratch layout: normalised rows (one FP32 copy, or the FP16 hi and lo
    // parts), then the similarity block [n_rows, round32(n)]
    const int64_t ld = (s.n + 31) / 32 * 32;
    const size_t row_bytes = farm::align256((size_t)n_rows * s.dim_pad * sizeof(float));
    const size_t n_row_copies = precision == FARM_PREC_FP32 ? 2 : 1;
    const size_t sim_bytes = farm::align256((size_t)n_rows * (size_t)ld * sizeof(float));
    if (n_rows > (int64_t)(farm::kScratchBytes / sizeof(float)) ||
        n_row_copies * row_bytes + sim_bytes > farm::kScratchBytes)
        return fail(FARM_EINVAL,
                    "farm_rank_rows_noalloc: n_rows x (scene objects + descriptor length) exceeds the "
                    "FARM_NOALLOC_SCRATCH_BYTES scratch array; split the rows into smaller calls");
    cudaError_t e = cudaSetDevice(c.device);
    if (e != cudaSuccess) return fail(FARM_ECUDA, cudaGetErrorString(e));
    if (c.device < 0 || c.device >= farm::kMaxDevices) return fail(FARM_EINVAL, "device ordinal out of range");
    void *base = nullptr;
    {
        std::lock_guard<std::mutex> lock(farm::g_setup_mutex);
        base = farm::g_scratch_ptr[c.device];
    }
    if (!base) return fail(FARM_ESTATE, "farm_rank_rows_noalloc: the scratch array was not set up by farm_create");
    unsigned char *b = static_cast<unsigned char *>(base);
    float *q0 = reinterpret_cast<float *>(b);
    float *q1 = n_row_copies == 2 ? reinterpret_cast<float *>(b + row_bytes) : nullptr;
    float *S = reinterpret_cast<float *>(b + n_row_copies * row_bytes);
    // every scratch entry read below is written earlier in this call: no clearing needed
    if (precision == FARM_PREC_FP32) {
        c.launches += 1;
        uint16_t *h0 = reinterpret_cast<uint16_t *>(q0), *h1 = reinterpret_cast<uint16_t *>(q1);
        e = farm::launch_normalize_rows(emb, nullptr, n_rows, s.dim, s.dim_pad, nullptr, h0, h1, nullptr, c.d_err,
                                        farm::kErrBadRow, c.stream);
        if (e != cudaSuccess) return fail(FARM_ECUDA, cudaGetErrorString(e));
        if (!farm::sim_tc_available()) return fail(FARM_EINVAL, "the tensor-core FP32 similarity path is not built");
        c.launches += 1;
        e = farm::launch_sim_tc_f16x3(h0, h1, s.desc_hi, s.desc_lo, S, n_rows, s.n, s.dim_pad, ld, nullptr, c.num_sms,
                                      c.d_err, c.stream);
    } else {
        c.launches += 1;
        e = farm::launch_normalize_rows(emb, nullptr, n_rows, s.dim, s.dim_pad, q0, nullptr, nullptr, nullptr,
                                        c.d_err, farm::kErrBadRow, c.stream);
        if (e != cudaSuccess) return fail(FARM_ECUDA, cudaGetErrorString(e));
        c.launches += 1;
        e = farm::launch_sim_simt(q0, s.desc32, S, n_rows, s.n, s.dim_pad, ld, c.stream);
    }
    if (e != cudaSuccess) return fail(FARM_ECUDA, cudaGetErrorString(e));
    c.launches += 1;
    e = farm::launch_select_rows(S, ld, s.n, n_rows, n_rows, r, 1, out_idx, out_cos, 0, r, nullptr, 0, 1, c.stream);
    if (e != cudaSuccess) return fail(FARM_ECUDA, cudaGetErrorString(e));
    return FARM_OK;
}
