"""ctypes binding of libfarm (include/farm.h), one function per C entry point.

Argument marshalling only: numpy arrays are host pointers, CUDA torch tensors
are device pointers (FARM_PTR_DEVICE); every step of the computation runs in
the library's kernels.  If libfarm.so is missing this module raises at import
time -- there is no other implementation to fall back to.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import _build

PREC_FP32 = 0
PREC_BF16 = 1
PREC_FP8 = 2
PREC_FP32_SIMT = 3
PREC_LEARNED = 4
PTR_DEVICE = 1
GRAPH = 2          # FARM_GRAPH
UNFUSED = 4        # FARM_UNFUSED
ASYNC = 8          # FARM_ASYNC
FUSED = 16         # FARM_FUSED
# predicate codes (farm_pred)
(ABOVE, BELOW, LEFT_OF, RIGHT_OF, NEAR, NEXT_TO, ON, IN_FRONT_OF, BEHIND, CLOSEST, FARTHEST, NEAR_H,
 INSIDE) = range(13)
N_STAGES = 4
STATUS = {0: "FARM_OK", 1: "FARM_EINVAL", 2: "FARM_ENOMEM", 3: "FARM_ECUDA", 4: "FARM_ESTATE",
          5: "FARM_ETIMEOUT"}


class FarmError(RuntimeError):
    def __init__(self, status: int, message: str):
        self.status = status
        super().__init__(f"{STATUS.get(status, status)}: {message}")


class FarmParams(C.Structure):
    _fields_ = [("mu", C.c_float), ("w", C.c_float), ("class_mis", C.c_float),
                ("sigma_near", C.c_float), ("tau_v", C.c_float), ("tau_h", C.c_float),
                ("z_min", C.c_float), ("k_anchor", C.c_int32), ("k_max", C.c_int32),
                ("rescore", C.c_int32), ("rescore_band", C.c_float), ("sigma_next", C.c_float),
                ("on_gate", C.c_float), ("on_band", C.c_float), ("tau_d", C.c_float),
                ("k_closest", C.c_int32)]


def _load():
    path = _build.LIB
    if not os.path.exists(path):
        raise ImportError(f"libfarm.so is not built ({path}); run __graft_entry__.build()")
    lib = C.CDLL(path)
    P, I32, I64, U32, U64 = C.c_void_p, C.c_int32, C.c_int64, C.c_uint32, C.c_uint64
    sig = {
        "farm_default_params": (None, [P]),
        "farm_create": (C.c_int, [P, C.c_int, P, P]),
        "farm_destroy": (C.c_int, [P]),
        "farm_memory_upload": (C.c_int, [P, I32, I64, I32, P, P, P, I32, P, U32]),
        "farm_query_batch": (C.c_int, [P, I64, P, P, P, P, P, P, I32, U32, P]),
        "farm_memory_add_space": (C.c_int, [P, I32, I32, I32, P, U32]),
        "farm_query_batch_rrf": (C.c_int, [P, I32, I64, I32, P, P, P, P, P, P, U32, P]),
        "farm_associate": (C.c_int, [P, I64, P, P, P, P, P, I64, P, P, P, I32, C.c_float, C.c_float, I32,
                                     P, P, P, P, P, P, P, P, U32]),
        "farm_topk": (C.c_int, [P, U64, I32, P, P, P, P, U32]),
        "farm_sync": (C.c_int, [P]),
        "farm_similarity": (C.c_int, [P, I32, I64, P, I32, P, U32]),
        "farm_scene_info": (C.c_int, [P, I32, P, P]),
        "farm_select_fallbacks": (C.c_int, [P, P, I32]),
        "farm_sim_tuning": (C.c_int, [P, P, I32, P]),
        "farm_sim_variant_pin": (C.c_int, [P, I32]),
        "farm_similarity_variant": (C.c_int, [P, I32, I64, P, I32, I32, P, U32]),
        "farm_candidates": (C.c_int, [P, U64, P, P, P, P]),
        "farm_rank_rows_noalloc": (C.c_int, [P, I32, I64, P, I32, I32, P, P]),
        "farm_mlp_set": (C.c_int, [P, I32, I32, I32, P, P, P, P]),
        "farm_mlp_get": (C.c_int, [P, P, P, P, P]),
        "farm_memory_release": (C.c_int, [P, I32]),
        "farm_mlp_loss_grad": (C.c_int, [P, I64, P, P, P, P, I32, P, P]),
        "farm_mlp_train": (C.c_int, [P, I32, P, I64, P, I64, P, P, P, P, P, I32, I32, C.c_float, U64, P]),
        "farm_mlp_embed": (C.c_int, [P, I64, P, I32, P]),
        "farm_set_profiling": (C.c_int, [P, I32]),
        "farm_stage_times": (C.c_int, [P, P, P, I32]),
        "farm_last_error": (C.c_char_p, [P]),
        "farm_version": (C.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_lib = _load()


def exported_symbols():
    return ["farm_default_params", "farm_create", "farm_destroy", "farm_memory_upload",
            "farm_query_batch", "farm_memory_add_space", "farm_query_batch_rrf", "farm_associate", "farm_topk", "farm_sync", "farm_similarity", "farm_scene_info",
            "farm_select_fallbacks", "farm_sim_tuning", "farm_sim_variant_pin", "farm_similarity_variant",
            "farm_candidates",
            "farm_rank_rows_noalloc", "farm_memory_release", "farm_mlp_set", "farm_mlp_get", "farm_mlp_loss_grad",
            "farm_mlp_train", "farm_mlp_embed", "farm_set_profiling", "farm_stage_times",
            "farm_last_error", "farm_version"]


def _is_cuda_tensor(x) -> bool:
    return hasattr(x, "is_cuda") and bool(x.is_cuda)


class _Arr:
    """A pointer plus the object that keeps its memory alive."""

    def __init__(self, x, dtype, name, allow_device=True):
        self.keep = None
        self.device = False
        if x is None:
            self.ptr = None
            return
        if _is_cuda_tensor(x):
            if not allow_device:
                raise FarmError(1, f"{name} must be host memory")
            import torch
            tdt = {np.float32: torch.float32, np.int32: torch.int32}[dtype]
            t = x if (x.dtype == tdt and x.is_contiguous()) else x.to(tdt).contiguous()
            self.keep = t
            self.ptr = C.c_void_p(t.data_ptr())
            self.device = True
            return
        if hasattr(x, "numpy") and not isinstance(x, np.ndarray):
            x = x.detach().cpu().numpy()
        a = np.ascontiguousarray(x, dtype=dtype)
        self.keep = a
        self.ptr = a.ctypes.data_as(C.c_void_p)


def _ck(ctx, st):
    if st != 0:
        msg = _lib.farm_last_error(ctx).decode() if ctx else ""
        raise FarmError(st, msg)


def _flags(*arrs):
    devs = {a.device for a in arrs if a.ptr is not None}
    if len(devs) > 1:
        raise FarmError(1, "mixing host and device arrays in one call")
    return PTR_DEVICE if devs == {True} else 0


def farm_version() -> str:
    return _lib.farm_version().decode()


def farm_default_params() -> FarmParams:
    p = FarmParams()
    _lib.farm_default_params(C.byref(p))
    return p


def farm_create(device: int = 0, stream=None, params: FarmParams | None = None):
    ctx = C.c_void_p()
    s = None if stream is None else C.c_void_p(int(getattr(stream, "cuda_stream", stream)))
    st = _lib.farm_create(C.byref(ctx), int(device), s, C.byref(params) if params else None)
    if st != 0:
        raise FarmError(st, "farm_create failed (bad params or no CUDA device)")
    return ctx


def farm_destroy(ctx) -> None:
    _ck(None, _lib.farm_destroy(ctx))


def farm_last_error(ctx) -> str:
    return _lib.farm_last_error(ctx).decode()


def farm_memory_upload(ctx, scene_id: int, desc, cls, box, views=None) -> None:
    d = _Arr(desc, np.float32, "desc")
    c = _Arr(cls, np.int32, "cls")
    b = _Arr(box, np.float32, "box")
    n, dim = (int(desc.shape[0]), int(desc.shape[1]))
    n_views = 0 if views is None else int(views.shape[1])
    v = _Arr(views if n_views > 0 else None, np.float32, "views")
    flags = _flags(d, c, b, v)
    _ck(ctx, _lib.farm_memory_upload(ctx, int(scene_id), n, dim, d.ptr, c.ptr, b.ptr, n_views,
                                     v.ptr, flags))


def farm_query_batch(ctx, scene_of_q, tgt_emb, tgt_cls, c_off, c_pred, c_emb,
                     precision: int = PREC_FP32, graph: bool = False, fused=None) -> int:
    """Enqueue a batch (see farm.h); graph=True passes FARM_GRAPH, fused=True
    FARM_FUSED and fused=False FARM_UNFUSED (None: the library's default)."""
    n_q = int(len(tgt_cls))
    s = _Arr(scene_of_q, np.int32, "scene_of_q", allow_device=False)
    tc = _Arr(tgt_cls, np.int32, "tgt_cls", allow_device=False)
    co = _Arr(c_off, np.int32, "c_off", allow_device=False)
    cp = _Arr(c_pred, np.int32, "c_pred", allow_device=False)
    te = _Arr(tgt_emb, np.float32, "tgt_emb")
    ce = _Arr(c_emb, np.float32, "c_emb")
    flags = _flags(te, ce) | (GRAPH if graph else 0) | ({None: 0, True: FUSED, False: UNFUSED}[fused])
    h = C.c_uint64()
    _ck(ctx, _lib.farm_query_batch(ctx, n_q, s.ptr, te.ptr, tc.ptr, co.ptr, cp.ptr, ce.ptr,
                                   int(precision), flags, C.byref(h)))
    return int(h.value)


class FarmChannel(C.Structure):
    _fields_ = [("space", C.c_int32), ("weight", C.c_float)]


def farm_memory_add_space(ctx, scene_id: int, space: int, desc) -> None:
    """Store descriptor space `space` (>= 1) of an uploaded scene (see farm.h)."""
    d = _Arr(desc, np.float32, "desc")
    _ck(ctx, _lib.farm_memory_add_space(ctx, int(scene_id), int(space), int(desc.shape[1]), d.ptr, _flags(d)))


def farm_query_batch_rrf(ctx, scene_id: int, channels, tgt_embs, tgt_cls, c_off, c_pred, c_embs) -> int:
    """Enqueue a fused batch over several channels (see farm.h).  channels:
    [(space, weight)]; tgt_embs / c_embs: either one [n_q, dim] / [n_c, dim]
    array per channel (all numpy, or all CUDA tensors; laid end to end for the
    call) or one flat FP32 array already laid out channel after channel."""
    n_q = int(len(tgt_cls))
    chs = (FarmChannel * len(channels))(*[FarmChannel(int(sp), float(w)) for sp, w in channels])

    def flat(xs):
        if not isinstance(xs, (list, tuple)):
            return xs
        if all(_is_cuda_tensor(x) for x in xs):
            import torch
            return torch.cat([x.reshape(-1).float() for x in xs])
        return np.concatenate([np.asarray(x, np.float32).ravel() for x in xs])
    tflat, cflat = flat(tgt_embs), flat(c_embs)
    te = _Arr(tflat, np.float32, "tgt_emb")
    ce = _Arr(cflat if len(cflat) else None, np.float32, "c_emb")
    tc = _Arr(tgt_cls, np.int32, "tgt_cls", allow_device=False)
    co = _Arr(c_off, np.int32, "c_off", allow_device=False)
    cp = _Arr(c_pred, np.int32, "c_pred", allow_device=False)
    h = C.c_uint64()
    _ck(ctx, _lib.farm_query_batch_rrf(ctx, int(scene_id), n_q, len(channels), chs, te.ptr, tc.ptr, co.ptr, cp.ptr,
                                       ce.ptr, _flags(te, ce), C.byref(h)))
    return int(h.value)


def farm_associate(ctx, ent, det, tau_f: float, h_max: float, max_m: int, out=None) -> dict:
    """Mapping-side association (see farm.h).  ent: dict(mu [3, N], cov [6, N],
    feat [N, F], active [N], w [N]); det: dict(mu [3, B], cov [6, B],
    feat [B, F]); all numpy, or all CUDA tensors (then `out` may hold CUDA
    tensors for the results)."""
    arrs = [_Arr(ent["mu"], np.float32, "ent_mu"), _Arr(ent["cov"], np.float32, "ent_cov"),
            _Arr(ent["feat"], np.float32, "ent_feat"), _Arr(ent["active"], np.int32, "ent_active"),
            _Arr(ent["w"], np.float32, "ent_w"), _Arr(det["mu"], np.float32, "det_mu"),
            _Arr(det["cov"], np.float32, "det_cov"), _Arr(det["feat"], np.float32, "det_feat")]
    N, B = int(ent["mu"].shape[1]), int(det["mu"].shape[1])
    F = int(ent["feat"].shape[1])
    T = N + B
    dev = _flags(*arrs) == PTR_DEVICE
    if out is None:
        if dev:
            import torch
            mk = lambda shape, dt: torch.empty(shape, dtype=dt, device="cuda")   # noqa: E731
            i32, f32 = torch.int32, torch.float32
        else:
            mk = lambda shape, dt: np.empty(shape, dtype=dt)   # noqa: E731
            i32, f32 = np.int32, np.float32
        out = dict(match_cnt=mk((B,), i32), match_idx=mk((B, max_m), i32), match_h=mk((B, max_m), f32),
                   parent=mk((T,), i32), w=mk((T,), f32), mu=mk((3, T), f32), cov=mk((6, T), f32),
                   feat=mk((T, F), f32))
    keys = ["match_cnt", "match_idx", "match_h", "parent", "w", "mu", "cov", "feat"]
    ptr = lambda x: C.c_void_p(x.data_ptr()) if _is_cuda_tensor(x) else x.ctypes.data_as(C.c_void_p)  # noqa: E731
    _ck(ctx, _lib.farm_associate(ctx, N, *[a.ptr for a in arrs[:5]], B, *[a.ptr for a in arrs[5:]], F,
                                 float(tau_f), float(h_max), int(max_m), *[ptr(out[k]) for k in keys],
                                 PTR_DEVICE if dev else 0))
    return out


def farm_topk(ctx, handle: int, k: int, n_q: int, out_idx=None, out_score=None, out_pred=None,
              out_anchor=None, breakdown: bool = True, asynchronous: bool = False):
    """TopK of a batch.  Without output arrays, returns new numpy arrays.
    asynchronous=True (host outputs): FARM_ASYNC, valid after the next farm_sync."""
    if out_idx is None:
        out_idx = np.zeros((n_q, k), np.int32)
        out_score = np.zeros((n_q, k), np.float32)
        if breakdown:
            out_pred = np.zeros((n_q, k, 4), np.float32)
            out_anchor = np.zeros((n_q, k, 4), np.int32)
    arrs = [out_idx, out_score, out_pred, out_anchor]
    dev = any(_is_cuda_tensor(a) for a in arrs if a is not None)
    for a in arrs:
        if a is None:
            continue
        if dev != _is_cuda_tensor(a):
            raise FarmError(1, "mixing host and device outputs")
        if not dev and not (isinstance(a, np.ndarray) and a.flags.c_contiguous):
            raise FarmError(1, "host outputs must be C-contiguous numpy arrays")
    ptr = (lambda a: None if a is None else C.c_void_p(a.data_ptr() if dev else a.ctypes.data))
    _ck(ctx, _lib.farm_topk(ctx, C.c_uint64(handle), int(k), ptr(out_idx), ptr(out_score),
                            ptr(out_pred), ptr(out_anchor),
                            PTR_DEVICE if dev else (ASYNC if asynchronous else 0)))
    return dict(idx=out_idx, score=out_score, pred=out_pred, anchor=out_anchor)


def farm_sync(ctx) -> None:
    _ck(ctx, _lib.farm_sync(ctx))


def farm_select_fallbacks(ctx, reset: bool = False) -> int:
    """Rows the thresholded select handed to its exact fallback (see farm.h)."""
    v = C.c_int64()
    _ck(ctx, _lib.farm_select_fallbacks(ctx, C.byref(v), 1 if reset else 0))
    return int(v.value)


def farm_sim_tuning(ctx):
    """The autotuner's decisions: a list of (mode, log2 rows, log2 mean objects per row, variant)."""
    n = C.c_int32()
    _ck(ctx, _lib.farm_sim_tuning(ctx, None, 0, C.byref(n)))
    buf = np.zeros((max(n.value, 1), 4), np.int32)
    _ck(ctx, _lib.farm_sim_tuning(ctx, buf.ctypes.data_as(C.c_void_p), n.value, C.byref(n)))
    return [tuple(int(x) for x in r) for r in buf[:n.value]]


def farm_sim_variant_pin(ctx, variant: int) -> None:
    """Pin the grouped similarity to one tile variant (0..2), or -1 for the autotuner."""
    _ck(ctx, _lib.farm_sim_variant_pin(ctx, int(variant)))


def farm_similarity_variant(ctx, scene_id: int, emb, precision: int, variant: int):
    """Cosines [rows, n] of `emb` against a scene by one tile variant (host arrays)."""
    e = np.ascontiguousarray(emb, dtype=np.float32)
    n_scene, _ = farm_scene_info(ctx, scene_id)
    out = np.zeros((e.shape[0], n_scene), np.float32)
    _ck(ctx, _lib.farm_similarity_variant(ctx, int(scene_id), int(e.shape[0]), e.ctypes.data_as(C.c_void_p),
                                          int(precision), int(variant), out.ctypes.data_as(C.c_void_p), 0))
    return out


def farm_scene_info(ctx, scene_id: int):
    """(n, dim) of an uploaded scene."""
    n = C.c_int64()
    dim = C.c_int32()
    _ck(ctx, _lib.farm_scene_info(ctx, int(scene_id), C.byref(n), C.byref(dim)))
    return int(n.value), int(dim.value)


def farm_similarity(ctx, scene_id: int, emb, n: int, precision: int = PREC_FP32, out=None):
    """Cosines [rows, n] of `emb` against scene `scene_id`; n must be the
    scene's object count (checked against the library's record)."""
    e = _Arr(emb, np.float32, "emb")
    rows = int(emb.shape[0])
    n_scene, _ = farm_scene_info(ctx, scene_id)
    if int(n) != n_scene:
        raise FarmError(1, f"n = {n} but scene {scene_id} holds {n_scene} objects")
    if out is None:
        out = np.zeros((rows, n), np.float32)
    if _is_cuda_tensor(out):
        import torch
        ok = out.dtype == torch.float32 and out.is_contiguous()
    else:
        ok = isinstance(out, np.ndarray) and out.dtype == np.float32 and out.flags["C_CONTIGUOUS"]
    if not ok or tuple(out.shape) != (rows, n):
        raise FarmError(1, f"out must be a contiguous FP32 array of shape ({rows}, {n})")
    dev = _is_cuda_tensor(out)
    if dev != e.device:
        raise FarmError(1, "emb and out must both be host or both be device")
    optr = C.c_void_p(out.data_ptr() if dev else out.ctypes.data)
    _ck(ctx, _lib.farm_similarity(ctx, int(scene_id), rows, e.ptr, int(precision), optr,
                                  PTR_DEVICE if dev else 0))
    return out


def farm_candidates(ctx, handle: int, n_q: int, n_c: int):
    r = C.c_int32()
    k = C.c_int32()
    _ck(ctx, _lib.farm_candidates(ctx, C.c_uint64(handle), None, None, C.byref(r), C.byref(k)))
    t = np.full((n_q, r.value), -1, np.int32)
    l = np.full((max(n_c, 0), k.value), -1, np.int32)
    _ck(ctx, _lib.farm_candidates(ctx, C.c_uint64(handle), t.ctypes.data_as(C.c_void_p),
                                  l.ctypes.data_as(C.c_void_p), None, None))
    return t, l


def farm_rank_rows_noalloc(ctx, scene_id: int, emb, r: int, precision: int, out_idx, out_cos=None):
    """Rank lists of device embedding rows with no allocation (CUDA tensors only)."""
    for name, t in (("emb", emb), ("out_idx", out_idx), ("out_cos", out_cos)):
        if t is not None and not _is_cuda_tensor(t):
            raise FarmError(1, f"{name} must be a CUDA tensor")
    e = _Arr(emb, np.float32, "emb")
    if not (out_idx.is_contiguous() and (out_cos is None or out_cos.is_contiguous())):
        raise FarmError(1, "outputs must be contiguous")
    _ck(ctx, _lib.farm_rank_rows_noalloc(ctx, int(scene_id), int(emb.shape[0]), e.ptr, int(r), int(precision),
                                         C.c_void_p(out_idx.data_ptr()),
                                         None if out_cos is None else C.c_void_p(out_cos.data_ptr())))
    return out_idx, out_cos


def _host(x, dtype):
    a = np.ascontiguousarray(x, dtype=dtype)
    return a, a.ctypes.data_as(C.c_void_p)


def farm_mlp_set(ctx, W1, b1, W2, b2) -> None:
    W1, p1 = _host(W1, np.float32)
    b1, p2 = _host(b1, np.float32)
    W2, p3 = _host(W2, np.float32)
    b2, p4 = _host(b2, np.float32)
    hidden, dim = W1.shape
    out_dim = W2.shape[0]
    _ck(ctx, _lib.farm_mlp_set(ctx, int(dim), int(hidden), int(out_dim), p1, p2, p3, p4))


def farm_mlp_get(ctx, dim: int, hidden: int, out_dim: int):
    W1 = np.zeros((hidden, dim), np.float32)
    b1 = np.zeros(hidden, np.float32)
    W2 = np.zeros((out_dim, hidden), np.float32)
    b2 = np.zeros(out_dim, np.float32)
    _ck(ctx, _lib.farm_mlp_get(ctx, W1.ctypes.data_as(C.c_void_p), b1.ctypes.data_as(C.c_void_p),
                               W2.ctypes.data_as(C.c_void_p), b2.ctypes.data_as(C.c_void_p)))
    return W1, b1, W2, b2


def farm_memory_release(ctx, scene_id: int) -> None:
    """Free an uploaded scene's device memory."""
    _ck(ctx, _lib.farm_memory_release(ctx, int(scene_id)))


def farm_mlp_loss_grad(ctx, xq, xd, y, w, n_params: int, precision: int = PREC_FP32_SIMT):
    """Loss and gradient of the prefilter network on host pairs, in FP32 on the
    CUDA cores (PREC_FP32_SIMT) or in the BF16 tensor-core training arithmetic (PREC_BF16)."""
    xq, pq = _host(xq, np.float32)
    xd, pd = _host(xd, np.float32)
    y, py = _host(y, np.float32)
    wp = None
    if w is not None:
        w, wp = _host(w, np.float32)
    loss = np.zeros(1, np.float32)
    grad = np.zeros(n_params, np.float32)
    _ck(ctx, _lib.farm_mlp_loss_grad(ctx, int(xq.shape[0]), pq, pd, py, wp, int(precision),
                                     loss.ctypes.data_as(C.c_void_p), grad.ctypes.data_as(C.c_void_p)))
    return float(loss[0]), grad


def farm_mlp_train(ctx, scene_id, rows, pair_row, pair_obj, y, w=None, epochs: int = 1,
                   batch: int = 4096, lr: float = 1e-3, seed: int = 0, pair_scene=None):
    """Train the prefilter; scene_id is one scene id, or a list of them with
    pair_scene[i] the position of pair i's scene in that list."""
    ids = [int(scene_id)] if np.isscalar(scene_id) else [int(x) for x in scene_id]
    sids, ps_ = _host(np.asarray(ids, np.int32), np.int32)
    rows, pr = _host(rows, np.float32)
    a, pa = _host(pair_row, np.int32)
    o, po = _host(pair_obj, np.int32)
    yy, py = _host(y, np.float32)
    wp = None
    if w is not None:
        ww, wp = _host(w, np.float32)
    psp = None
    if pair_scene is not None:
        psa, psp = _host(pair_scene, np.int32)
    losses = np.zeros(epochs, np.float32)
    _ck(ctx, _lib.farm_mlp_train(ctx, len(ids), ps_, int(rows.shape[0]), pr, int(a.shape[0]), pa, psp, po, py, wp,
                                 int(epochs), int(batch), C.c_float(lr), C.c_uint64(seed),
                                 losses.ctypes.data_as(C.c_void_p)))
    return losses


def farm_mlp_embed(ctx, x, out_dim: int, precision: int = PREC_FP32_SIMT):
    x, px = _host(x, np.float32)
    out = np.zeros((x.shape[0], out_dim), np.float32)
    _ck(ctx, _lib.farm_mlp_embed(ctx, int(x.shape[0]), px, int(precision), out.ctypes.data_as(C.c_void_p)))
    return out


def farm_set_profiling(ctx, on: bool) -> None:
    _ck(ctx, _lib.farm_set_profiling(ctx, 1 if on else 0))


def farm_stage_times(ctx, reset: bool = True):
    ms = (C.c_float * N_STAGES)()
    n = C.c_int64()
    _ck(ctx, _lib.farm_stage_times(ctx, ms, C.byref(n), 1 if reset else 0))
    return list(ms), int(n.value)
