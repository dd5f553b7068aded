"""ctypes binding of the FP64 oracle in farm_oracle.c (test infrastructure).

`build()` compiles the C file with gcc (OpenMP) into oracle/_build/; every
function below marshals numpy arrays into the C calls and nothing else.
"""
from __future__ import annotations

import ctypes as C
import dataclasses
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "farm_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")

(ABOVE, BELOW, LEFT_OF, RIGHT_OF, NEAR, NEXT_TO, ON, IN_FRONT_OF, BEHIND, CLOSEST, FARTHEST, NEAR_H,
 INSIDE, BETWEEN, BETWEEN_AND) = range(15)


@dataclasses.dataclass
class OracleParams:
    """The method's constants (App. D.2): RRF offset mu = 5, blend weight
    w = 0.5, class-mismatch factor 0.3, Near width 0.5 m, NextTo width 1.0 m;
    tau_v, tau_h, z_min, the On gate and band widths, tau_d and the size of
    the Closest/Farthest candidate set are not given by the paper (readings)."""
    mu: float = 5.0
    w: float = 0.5
    class_mis: float = 0.3
    sigma_near: float = 0.5
    tau_v: float = 0.25
    tau_h: float = 0.10
    z_min: float = 0.05
    k_anchor: int = 16
    sigma_next: float = 1.0
    on_gate: float = 0.10
    on_band: float = 0.10
    tau_d: float = 0.25
    k_closest: int = 16


class _Params(C.Structure):
    _fields_ = [("mu", C.c_double), ("w", C.c_double), ("class_mis", C.c_double),
                ("sigma_near", C.c_double), ("tau_v", C.c_double), ("tau_h", C.c_double),
                ("z_min", C.c_double), ("k_anchor", C.c_int64), ("sigma_next", C.c_double),
                ("on_gate", C.c_double), ("on_band", C.c_double), ("tau_d", C.c_double),
                ("k_closest", C.c_int64)]


class _Scene(C.Structure):
    _fields_ = [("n", C.c_int64), ("dim", C.c_int64), ("desc", C.c_void_p),
                ("cls", C.c_void_p), ("box", C.c_void_p), ("n_views", C.c_int64),
                ("views", C.c_void_p)]


def build(force: bool = False) -> str:
    """Compile farm_oracle.c into a shared library (gcc, -O2, OpenMP).

    FARM_ORACLE_LIB names a prebuilt library to use instead (the mutation
    tests point it at copies of the oracle with planted mistakes)."""
    alt = os.environ.get("FARM_ORACLE_LIB")
    if alt:
        return alt
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", "-Wall",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


_lib = None


def load():
    global _lib
    if _lib is None:
        lib = C.CDLL(build())
        P = C.c_void_p
        lib.orc_sigmoid.restype = C.c_double
        lib.orc_sigmoid.argtypes = [C.c_double]
        lib.orc_relation.restype = C.c_double
        lib.orc_relation.argtypes = [P, P, C.c_int32, C.c_int64, C.c_int64]
        lib.orc_relation_in.restype = C.c_double
        lib.orc_relation_in.argtypes = [P, P, C.c_int32, C.c_int64, C.c_int64, P, C.c_int64]
        lib.orc_cosines.restype = C.c_int
        lib.orc_cosines.argtypes = [P, P, P]
        lib.orc_ranks.restype = C.c_int
        lib.orc_ranks.argtypes = [C.c_int64, P, P]
        lib.orc_query_all.restype = C.c_int
        lib.orc_query_all.argtypes = [P, P, P, C.c_int32, C.c_int32, P, P, P, P, P, P, P, P]
        lib.orc_topk.restype = C.c_int
        lib.orc_topk.argtypes = [C.c_int64, P, C.c_int64, P]
        lib.orc_batch.restype = C.c_int
        lib.orc_batch.argtypes = [P, P, C.c_int64, P, P, P, P, P, C.c_int64, P, P, P, P, C.c_int32]
        lib.orc_query_bounds.restype = C.c_int
        lib.orc_query_bounds.argtypes = [P, P, P, C.c_int32, C.c_int32, P, P, C.c_double,
                                         P, P, P, P, P, P, P]
        lib.orc_query_mc.restype = C.c_int
        lib.orc_query_mc.argtypes = [P, P, C.c_int32, P, C.c_int32, P, P, P, C.c_int32, C.c_int32, P, P,
                                     P, P, P, P, P]
        lib.orc_query_bounds_mc.restype = C.c_int
        lib.orc_query_bounds_mc.argtypes = [P, P, C.c_int32, P, C.c_int32, P, P, P, C.c_int32, C.c_int32, P,
                                            P, C.c_double, P, P, P, P, P, P, P]
        lib.orc_between.restype = C.c_double
        lib.orc_between.argtypes = [P, P, C.c_int64, C.c_int64, C.c_int64]
        lib.orc_hellinger.restype = C.c_double
        lib.orc_hellinger.argtypes = [P, P, P, P]
        lib.orc_associate.restype = C.c_int
        lib.orc_associate.argtypes = [C.c_int64, P, P, P, P, P, C.c_int64, P, P, P, C.c_int64, C.c_double,
                                      C.c_double, C.c_int64, P, P, P, P, P, P, P, P]
        lib.orc_num_threads.restype = C.c_int
        lib.orc_num_threads.argtypes = []
        _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


class _SceneRef:
    """Holds contiguous copies of a synth.Scene's arrays alive for a call."""

    def __init__(self, scene):
        self.desc = np.ascontiguousarray(scene.desc, dtype=np.float32)
        self.cls = np.ascontiguousarray(scene.cls, dtype=np.int32)
        self.box = np.ascontiguousarray(scene.box, dtype=np.float32)
        self.views = np.ascontiguousarray(scene.views, dtype=np.float32)
        n, dim = self.desc.shape
        self.n = n
        self.dim = dim
        self.c = _Scene(n, dim, _ptr(self.desc), _ptr(self.cls), _ptr(self.box),
                        int(self.views.shape[1]), _ptr(self.views))


def _params(p: OracleParams | None):
    p = p or OracleParams()
    return _Params(p.mu, p.w, p.class_mis, p.sigma_near, p.tau_v, p.tau_h, p.z_min, p.k_anchor,
                   p.sigma_next, p.on_gate, p.on_band, p.tau_d, p.k_closest)


def _check(rc, what):
    if rc != 0:
        raise ValueError(f"oracle {what} failed with code {rc}")


def num_threads() -> int:
    return int(load().orc_num_threads())


def sigmoid(x: float) -> float:
    return float(load().orc_sigmoid(float(x)))


def relation(scene, pred: int, e: int, a: int, params: OracleParams | None = None) -> float:
    sr, pp = _SceneRef(scene), _params(params)
    return float(load().orc_relation(C.byref(sr.c), C.byref(pp), int(pred), int(e), int(a)))


def between(scene, e: int, ap: int, aq: int, params: OracleParams | None = None) -> float:
    """The Between relation of e to the landmark pair (a_p, a_q)."""
    sr, pp = _SceneRef(scene), _params(params)
    return float(load().orc_between(C.byref(sr.c), C.byref(pp), int(e), int(ap), int(aq)))


def relation_in(scene, pred: int, e: int, a: int, cand_set, params: OracleParams | None = None) -> float:
    """r_rho(e, a) with the Closest/Farthest candidate set given explicitly."""
    sr, pp = _SceneRef(scene), _params(params)
    cs = np.ascontiguousarray(cand_set, dtype=np.int64)
    return float(load().orc_relation_in(C.byref(sr.c), C.byref(pp), int(pred), int(e), int(a),
                                        _ptr(cs if cs.size else np.zeros(1, np.int64)), int(cs.size)))


def cosines(scene, u) -> np.ndarray:
    sr = _SceneRef(scene)
    u = np.ascontiguousarray(u, dtype=np.float32)
    out = np.zeros(sr.n, np.float64)
    _check(load().orc_cosines(C.byref(sr.c), _ptr(u), _ptr(out)), "cosines")
    return out


def ranks(c) -> np.ndarray:
    c = np.ascontiguousarray(c, dtype=np.float64)
    out = np.zeros(c.shape[0], np.int64)
    _check(load().orc_ranks(c.shape[0], _ptr(c), _ptr(out)), "ranks")
    return out


def topk(s, k: int) -> np.ndarray:
    s = np.ascontiguousarray(s, dtype=np.float64)
    out = np.zeros(k, np.int64)
    _check(load().orc_topk(s.shape[0], _ptr(s), int(k), _ptr(out)), "topk")
    return out


def query_all(scene, u0, c_t, preds, u_c, params: OracleParams | None = None) -> dict:
    """Every intermediate of one query over all objects (steps 1-7)."""
    sr, pp = _SceneRef(scene), _params(params)
    preds = np.ascontiguousarray(preds, dtype=np.int32)
    m = int(preds.shape[0])
    u0 = np.ascontiguousarray(u0, dtype=np.float32)
    u_c = np.ascontiguousarray(np.asarray(u_c, dtype=np.float32).reshape(m, sr.dim))
    n = sr.n
    out = dict(cos0=np.zeros(n), rank0=np.zeros(n, np.int64), s_sem=np.zeros(n),
               t=np.zeros((m, n)), anchor=np.zeros((m, n), np.int64), s=np.zeros(n))
    rc = load().orc_query_all(C.byref(sr.c), C.byref(pp), _ptr(u0), int(c_t), m, _ptr(preds),
                              _ptr(u_c), _ptr(out["cos0"]), _ptr(out["rank0"]), _ptr(out["s_sem"]),
                              _ptr(out["t"]), _ptr(out["anchor"]), _ptr(out["s"]))
    _check(rc, "query_all")
    return out


def query_bounds(scene, u0, c_t, preds, u_c, tau: float,
                 params: OracleParams | None = None) -> dict:
    """Tie-tolerant bounds on what any result with cosine error <= tau/2 may score."""
    sr, pp = _SceneRef(scene), _params(params)
    preds = np.ascontiguousarray(preds, dtype=np.int32)
    m = int(preds.shape[0])
    u0 = np.ascontiguousarray(u0, dtype=np.float32)
    u_c = np.ascontiguousarray(np.asarray(u_c, dtype=np.float32).reshape(m, sr.dim))
    n = sr.n
    out = dict(s_lo=np.zeros(n), s_hi=np.zeros(n), t_lo=np.zeros((m, n)), t_hi=np.zeros((m, n)),
               rank_lo=np.zeros(n, np.int64), rank_hi=np.zeros(n, np.int64),
               in_p=np.zeros((m, n), np.int8))
    rc = load().orc_query_bounds(C.byref(sr.c), C.byref(pp), _ptr(u0), int(c_t), m, _ptr(preds),
                                 _ptr(u_c), float(tau), _ptr(out["s_lo"]), _ptr(out["s_hi"]),
                                 _ptr(out["t_lo"]), _ptr(out["t_hi"]), _ptr(out["rank_lo"]),
                                 _ptr(out["rank_hi"]), _ptr(out["in_p"]))
    _check(rc, "query_bounds")
    return out


def batch(scene, qb, k: int, params: OracleParams | None = None, n_threads: int = 0) -> dict:
    """TopK of every query in `qb` against one scene (OpenMP over queries)."""
    sr, pp = _SceneRef(scene), _params(params)
    n_q = qb.n_q
    tgt = np.ascontiguousarray(qb.tgt_emb, dtype=np.float32)
    tcls = np.ascontiguousarray(qb.tgt_cls, dtype=np.int32)
    coff = np.ascontiguousarray(qb.c_off, dtype=np.int32)
    cpred = np.ascontiguousarray(qb.c_pred, dtype=np.int32)
    cemb = np.ascontiguousarray(qb.c_emb, dtype=np.float32)
    out = dict(idx=np.zeros((n_q, k), np.int64), score=np.zeros((n_q, k)),
               t=np.zeros((n_q, k, 4)), anchor=np.zeros((n_q, k, 4), np.int64))
    rc = load().orc_batch(C.byref(sr.c), C.byref(pp), n_q, _ptr(tgt), _ptr(tcls), _ptr(coff),
                          _ptr(cpred), _ptr(cemb if cemb.size else np.zeros(1, np.float32)),
                          int(k), _ptr(out["idx"]), _ptr(out["score"]), _ptr(out["t"]),
                          _ptr(out["anchor"]), int(n_threads))
    _check(rc, "batch")
    return out


class _Space(C.Structure):
    _fields_ = [("dim", C.c_int64), ("desc", C.c_void_p)]


class _SpacesRef:
    """Contiguous float32 copies of a scene's descriptor spaces (a list of
    [n, dim_s] arrays) and the C table pointing at them."""

    def __init__(self, spaces):
        self.arrs = [np.ascontiguousarray(d, dtype=np.float32) for d in spaces]
        self.table = (_Space * len(self.arrs))(*[_Space(a.shape[1], _ptr(a)) for a in self.arrs])
        self.n = len(self.arrs)


def _mc_args(spaces, channels, u0, u_c, m):
    """channels: list of (space, weight); u0: list of per-channel target
    embeddings; u_c: list of per-channel [m, dim] landmark embeddings."""
    sp = _SpacesRef(spaces)
    ch_space = np.ascontiguousarray([c[0] for c in channels], dtype=np.int32)
    ch_w = np.ascontiguousarray([c[1] for c in channels], dtype=np.float64)
    u0f = np.ascontiguousarray(np.concatenate([np.asarray(x, np.float32).ravel() for x in u0]))
    ucf = np.ascontiguousarray(np.concatenate([np.asarray(x, np.float32).reshape(m, -1).ravel() for x in u_c])
                               if m > 0 else np.zeros(1, np.float32))
    return sp, ch_space, ch_w, u0f, ucf


def query_mc(scene, spaces, channels, u0, c_t, preds, u_c, params: OracleParams | None = None) -> dict:
    """One query over several retrieval channels (reciprocal-rank fusion,
    App. D.2 step 3): every intermediate over all objects."""
    sr, pp = _SceneRef(scene), _params(params)
    preds = np.ascontiguousarray(preds, dtype=np.int32)
    m = int(preds.shape[0])
    sp, chs, chw, u0f, ucf = _mc_args(spaces, channels, u0, u_c, m)
    n = sr.n
    out = dict(fused=np.zeros(n), s_sem=np.zeros(n), t=np.zeros((m, n)), anchor=np.zeros((m, n), np.int64),
               s=np.zeros(n))
    rc = load().orc_query_mc(C.byref(sr.c), sp.table, sp.n, C.byref(pp), len(channels), _ptr(chs), _ptr(chw),
                             _ptr(u0f), int(c_t), m, _ptr(preds if m else np.zeros(1, np.int32)), _ptr(ucf),
                             _ptr(out["fused"]), _ptr(out["s_sem"]), _ptr(out["t"]), _ptr(out["anchor"]),
                             _ptr(out["s"]))
    _check(rc, "query_mc")
    return out


def query_bounds_mc(scene, spaces, channels, u0, c_t, preds, u_c, tau: float,
                    params: OracleParams | None = None) -> dict:
    """Tie-tolerant bounds of query_mc (cosine error <= tau/2 in every channel)."""
    sr, pp = _SceneRef(scene), _params(params)
    preds = np.ascontiguousarray(preds, dtype=np.int32)
    m = int(preds.shape[0])
    sp, chs, chw, u0f, ucf = _mc_args(spaces, channels, u0, u_c, m)
    n = sr.n
    out = dict(s_lo=np.zeros(n), s_hi=np.zeros(n), t_lo=np.zeros((m, n)), t_hi=np.zeros((m, n)),
               F_lo=np.zeros(n), F_hi=np.zeros(n), in_p=np.zeros((m, n), np.int8))
    rc = load().orc_query_bounds_mc(C.byref(sr.c), sp.table, sp.n, C.byref(pp), len(channels), _ptr(chs),
                                    _ptr(chw), _ptr(u0f), int(c_t), m, _ptr(preds if m else np.zeros(1, np.int32)),
                                    _ptr(ucf), float(tau), _ptr(out["s_lo"]), _ptr(out["s_hi"]), _ptr(out["t_lo"]),
                                    _ptr(out["t_hi"]), _ptr(out["F_lo"]), _ptr(out["F_hi"]), _ptr(out["in_p"]))
    _check(rc, "query_bounds_mc")
    return out


def hellinger(mu1, cov1, mu2, cov2) -> float:
    """Hellinger distance of two 3D Gaussians (covariances packed xx, xy, xz, yy, yz, zz)."""
    a = [np.ascontiguousarray(x, dtype=np.float64) for x in (mu1, cov1, mu2, cov2)]
    return float(load().orc_hellinger(*[_ptr(x) for x in a]))


def associate(ent, det, tau_f: float, h_max: float, max_m: int) -> dict:
    """Mapping-side association of a detection batch with the entities
    (neighbour search, union-find correspondence, sufficient-statistics
    fusion).  ent: dict(mu [3, N], cov [6, N], feat [N, F], active [N], w [N]);
    det: dict(mu [3, B], cov [6, B], feat [B, F])."""
    f32 = lambda x: np.ascontiguousarray(x, dtype=np.float32)   # noqa: E731
    emu, ecov, efeat, ew = f32(ent["mu"]), f32(ent["cov"]), f32(ent["feat"]), f32(ent["w"])
    eact = np.ascontiguousarray(ent["active"], dtype=np.int32)
    dmu, dcov, dfeat = f32(det["mu"]), f32(det["cov"]), f32(det["feat"])
    N, B, F = emu.shape[1], dmu.shape[1], efeat.shape[1] if efeat.size else dfeat.shape[1]
    T = N + B
    out = dict(match_cnt=np.zeros(B, np.int64), match_idx=np.zeros((B, max_m), np.int64),
               match_h=np.zeros((B, max_m)), parent=np.zeros(T, np.int64), w=np.zeros(T),
               mu=np.zeros((3, T)), cov=np.zeros((6, T)), feat=np.zeros((T, F)))
    one = lambda a: _ptr(a if a.size else np.zeros(1, a.dtype))   # noqa: E731
    rc = load().orc_associate(N, one(emu), one(ecov), one(efeat), one(eact), one(ew), B, one(dmu), one(dcov),
                              one(dfeat), F, float(tau_f), float(h_max), int(max_m), one(out["match_cnt"]),
                              one(out["match_idx"]), one(out["match_h"]), one(out["parent"]), one(out["w"]),
                              one(out["mu"]), one(out["cov"]), one(out["feat"]))
    _check(rc, "associate")
    return out
