"""Seeded synthetic object memories and relational queries.

The shapes follow the paper's workloads (Sec. 3.1, App. E data card, App. F.1):
scenes of 10^1 to 10^4 m^2 holding tens to tens of thousands of objects, object
descriptors drawn around class centroids, each object seen from a ring of stored
camera views, and queries made of a target description plus 0-4 relational
constraints, each naming a predicate and a landmark description.

Only sampling and array layout live here.  Nothing in this file scores,
ranks or evaluates a predicate: planting a landmark uses plain coordinate
comparisons (is the landmark lower, higher, within a radius), not the
retrieval method's soft evaluators.

Layouts (shared by the oracle and the C-ABI):
  desc   float32 [n, dim]        row-major, unit norm (renormalised after noise)
  cls    int32   [n]
  box    float32 [6, n]          SoA rows cx, cy, cz, sx, sy, sz (metres, z up)
  views  float32 [6, V, n]       SoA rows ox, oy, oz, fx, fy, fz per view
  queries: tgt_emb float32 [n_q, dim] (not normalised), tgt_cls int32 [n_q],
           c_off int32 [n_q+1] (CSR), c_pred int32 [n_c], c_emb float32 [n_c, dim]
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

# Predicate codes of the C-ABI (include/farm.h): above, below, left_of,
# right_of, near.
N_PRED = 5          # the predicates of the benchmark workloads (codes 0-4)
N_PRED_ALL = 15     # with NextTo, On, InFrontOf, Behind, Closest, Farthest, NearH, Inside, Between (5-14)


@dataclasses.dataclass
class Scene:
    desc: np.ndarray          # [n, dim] float32
    cls: np.ndarray           # [n] int32
    box: np.ndarray           # [6, n] float32
    views: np.ndarray         # [6, V, n] float32
    centroids: np.ndarray | None = None   # [n_classes, dim] float64 (generator state)
    extent: tuple = (0.0, 0.0, 0.0)
    noise_sigma: float = 0.0

    @property
    def n(self) -> int:
        return int(self.desc.shape[0])

    @property
    def dim(self) -> int:
        return int(self.desc.shape[1])

    @property
    def n_views(self) -> int:
        return int(self.views.shape[1])

    @property
    def centers(self) -> np.ndarray:
        return self.box[:3].T


@dataclasses.dataclass
class QueryBatch:
    tgt_emb: np.ndarray       # [n_q, dim] float32
    tgt_cls: np.ndarray       # [n_q] int32, -1 = no class
    c_off: np.ndarray         # [n_q+1] int32
    c_pred: np.ndarray        # [n_c] int32
    c_emb: np.ndarray         # [n_c, dim] float32
    scene_of_q: np.ndarray    # [n_q] int32
    planted: np.ndarray | None = None    # [n_q] int64, planted target object
    planted_lm: np.ndarray | None = None  # [n_c] int64, planted landmark objects

    @property
    def n_q(self) -> int:
        return int(self.tgt_emb.shape[0])

    @property
    def n_c(self) -> int:
        return int(self.c_pred.shape[0])

    def subset(self, qs) -> "QueryBatch":
        qs = np.asarray(qs, dtype=np.int64)
        offs = self.c_off.astype(np.int64)
        rows = [np.arange(offs[q], offs[q + 1]) for q in qs]
        cat = np.concatenate(rows) if rows else np.zeros(0, np.int64)
        m = np.array([len(r) for r in rows], dtype=np.int64)
        c_off = np.zeros(len(qs) + 1, np.int32)
        c_off[1:] = np.cumsum(m)
        return QueryBatch(
            tgt_emb=np.ascontiguousarray(self.tgt_emb[qs]),
            tgt_cls=np.ascontiguousarray(self.tgt_cls[qs]),
            c_off=c_off,
            c_pred=np.ascontiguousarray(self.c_pred[cat]),
            c_emb=np.ascontiguousarray(self.c_emb[cat]).reshape(len(cat), self.tgt_emb.shape[1]),
            scene_of_q=np.ascontiguousarray(self.scene_of_q[qs]),
            planted=None if self.planted is None else self.planted[qs],
            planted_lm=None if self.planted_lm is None else self.planted_lm[cat],
        )


def _unit_rows(x: np.ndarray) -> np.ndarray:
    return x / np.linalg.norm(x, axis=1, keepdims=True)


def ring_views(centers: np.ndarray, n_views: int, rng: np.random.Generator,
               radius: float = 2.0, arc_deg: float = 120.0) -> np.ndarray:
    """V camera poses on a horizontal ring around each object centre.

    Cameras sit at the object's centre height, `radius` metres away, evenly
    spaced over an arc of `arc_deg` degrees starting at a random phase (the
    stretch of a robot's path from which it saw the object), each looking at
    the centre (z up).  A full 360-degree arc makes view-averaged left/right
    nearly symmetric, so the default is a partial arc.
    Returns float32 [6, V, n].
    """
    n = centers.shape[0]
    phase = rng.uniform(0.0, 2.0 * math.pi, size=n)
    views = np.zeros((6, n_views, n), dtype=np.float64)
    step = math.radians(arc_deg) / max(n_views - 1, 1) if arc_deg < 360.0 else 2.0 * math.pi / max(n_views, 1)
    for v in range(n_views):
        th = phase + step * v
        dx, dy = np.cos(th), np.sin(th)
        views[0, v] = centers[:, 0] + radius * dx
        views[1, v] = centers[:, 1] + radius * dy
        views[2, v] = centers[:, 2]
        views[3, v] = -dx
        views[4, v] = -dy
        views[5, v] = 0.0
    return views.astype(np.float32)


def make_scene(seed: int, n: int, dim: int, extent=(10.0, 10.0, 3.0),
               n_classes: int = 16, n_views: int = 4,
               distractor_classes: int = 0, distractor_frac: float = 0.0,
               noise: str = "scaled", noise_scale: float = 0.15) -> Scene:
    """One object memory.

    Box centres are uniform in the extent; box sizes are lognormal(-1, 0.5) per
    axis.  Each object belongs to a class; its descriptor is the class's unit
    Gaussian centroid plus isotropic noise, renormalised.  `noise="scaled"`
    draws per-dimension sigma = noise_scale/sqrt(dim) (noise norm about
    noise_scale); `noise="literal"` draws per-dimension sigma = noise_scale.
    With `distractor_classes` > 0, a fraction `distractor_frac` of the objects
    is spread evenly over that many classes (dense look-alike groups); the
    rest is uniform over the remaining classes.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    ext = np.asarray(extent, dtype=np.float64)
    centers = rng.uniform(0.0, 1.0, size=(n, 3)) * ext
    sizes = rng.lognormal(-1.0, 0.5, size=(n, 3))
    centroids = _unit_rows(rng.standard_normal((n_classes, dim)))
    if distractor_classes > 0:
        n_dis = int(round(distractor_frac * n))
        dis = np.arange(n_dis) % distractor_classes
        rest = distractor_classes + rng.integers(0, n_classes - distractor_classes, size=n - n_dis)
        cls = np.concatenate([dis, rest])
        cls = cls[rng.permutation(n)]
    else:
        cls = rng.integers(0, n_classes, size=n)
    sigma = noise_scale / math.sqrt(dim) if noise == "scaled" else noise_scale
    desc = centroids[cls] + sigma * rng.standard_normal((n, dim))
    desc = _unit_rows(desc).astype(np.float32)
    views = ring_views(centers, n_views, rng)
    box = np.concatenate([centers.T, sizes.T], axis=0).astype(np.float32)
    return Scene(desc=np.ascontiguousarray(desc), cls=cls.astype(np.int32),
                 box=np.ascontiguousarray(box), views=np.ascontiguousarray(views),
                 centroids=centroids, extent=tuple(float(e) for e in ext),
                 noise_sigma=sigma)


def _plant_landmark(rng, centers, e, pred, tree, radius=5.0, sizes=None):
    """Pick a landmark object for constraint `pred` on planted target `e`.

    Prefers objects within `radius` metres; among them, for above (0) a lower
    centre, for below (1) a higher centre, for near (4) one within 1 m, for
    next_to (5) one within 2 m, for on (6) a lower centre within 1 m
    horizontally, for near_h (11) one within 1 m, for inside (12) the
    largest box within 1 m; for the others any neighbour.  Falls back to any other
    object.
    `tree` is a KD-tree over the centres (neighbour lookup only).
    """
    n = centers.shape[0]
    cand = np.asarray(sorted(tree.query_ball_point(centers[e], radius)), dtype=np.int64)
    cand = cand[cand != e]
    if cand.size == 0:
        others = np.flatnonzero(np.arange(n) != e)
        return int(rng.choice(others)) if others.size else int(e)
    if pred == 0:
        pref = cand[centers[cand, 2] < centers[e, 2]]
    elif pred == 1:
        pref = cand[centers[cand, 2] > centers[e, 2]]
    elif pred == 4:
        d = centers[cand] - centers[e]
        pref = cand[np.einsum("ij,ij->i", d, d) <= 1.0]
    elif pred == 5:
        d = centers[cand] - centers[e]
        pref = cand[np.einsum("ij,ij->i", d, d) <= 4.0]
    elif pred == 6:
        d = centers[cand, :2] - centers[e, :2]
        pref = cand[(np.einsum("ij,ij->i", d, d) <= 1.0) & (centers[cand, 2] < centers[e, 2])]
    elif pred == 11:
        d = centers[cand] - centers[e]
        pref = cand[np.einsum("ij,ij->i", d, d) <= 1.0]
    elif pred == 12 and sizes is not None:
        d = centers[cand] - centers[e]
        near = cand[np.einsum("ij,ij->i", d, d) <= 1.0]
        pref = near[np.argsort(-np.prod(sizes[near], axis=1), kind="stable")[:1]] if near.size else near
    else:
        pref = cand
    pool = pref if pref.size else cand
    return int(rng.choice(pool))


def make_queries(seed: int, scene: Scene, n_q: int, m_choices=(2,),
                 distractor_classes: int = 0, distractor_target_frac: float = 0.0,
                 scene_id: int = 0, with_class: bool = True, preds=None) -> QueryBatch:
    """Relational queries with a planted target and planted landmarks.

    Each query plants a target object e*; its target embedding is the
    centroid of e*'s class plus the scene's descriptor noise (not
    renormalised), and its target class is e*'s class (or -1 when
    `with_class` is False).  The number of constraints is drawn uniformly from
    `m_choices`; each constraint draws a predicate uniformly from the five of
    the benchmark workloads (or from `preds`, a list of predicate codes) and
    plants a landmark near e* (see `_plant_landmark`); the landmark embedding
    is its class centroid plus noise.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    n, dim = scene.n, scene.dim
    centers = scene.centers.astype(np.float64)
    sizes = np.abs(scene.box[3:].T.astype(np.float64))
    cent = scene.centroids
    sigma = scene.noise_sigma
    if distractor_classes > 0:
        dis_objs = np.flatnonzero(scene.cls < distractor_classes)
        oth_objs = np.flatnonzero(scene.cls >= distractor_classes)
    m_choices = np.asarray(m_choices, dtype=np.int64)
    targets = np.zeros(n_q, np.int64)
    ms = rng.choice(m_choices, size=n_q)
    for q in range(n_q):
        if distractor_classes > 0 and rng.uniform() < distractor_target_frac and dis_objs.size:
            targets[q] = rng.choice(dis_objs)
        elif distractor_classes > 0 and oth_objs.size:
            targets[q] = rng.choice(oth_objs)
        else:
            targets[q] = rng.integers(0, n)
    tgt_emb = cent[scene.cls[targets]] + sigma * rng.standard_normal((n_q, dim))
    c_off = np.zeros(n_q + 1, np.int32)
    c_off[1:] = np.cumsum(ms)
    n_c = int(c_off[-1])
    pred_set = preds
    preds = rng.integers(0, N_PRED, size=n_c) if pred_set is None else rng.choice(np.asarray(pred_set), size=n_c)
    if pred_set is not None and (13 in pred_set or 14 in pred_set):
        # Between takes two consecutive constraints (13 then 14); a 13 with no
        # room after it, or a 14 without its 13, becomes near (4)
        for q in range(n_q):
            c, c1 = int(c_off[q]), int(c_off[q + 1])
            while c < c1:
                if preds[c] == 13 and c + 1 < c1:
                    preds[c + 1] = 14
                    c += 2
                    continue
                if preds[c] in (13, 14):
                    preds[c] = 4
                c += 1
    lms = np.zeros(n_c, np.int64)
    from scipy.spatial import cKDTree
    tree = cKDTree(centers)
    for q in range(n_q):
        for c in range(c_off[q], c_off[q + 1]):
            if preds[c] == 14:
                # the second landmark of a Between: the object nearest the far
                # side of the target from the first one
                far = 2.0 * centers[targets[q]] - centers[lms[c - 1]]
                _, near_idx = tree.query(far, k=min(4, n))
                near_idx = [int(j) for j in np.atleast_1d(near_idx) if j != targets[q] and j != lms[c - 1]]
                lms[c] = near_idx[0] if near_idx else int(lms[c - 1])
                continue
            lms[c] = _plant_landmark(rng, centers, int(targets[q]), int(preds[c]), tree, sizes=sizes)
    c_emb = cent[scene.cls[lms]] + sigma * rng.standard_normal((n_c, dim))
    tgt_cls = scene.cls[targets].astype(np.int32) if with_class else np.full(n_q, -1, np.int32)
    return QueryBatch(tgt_emb=np.ascontiguousarray(tgt_emb.astype(np.float32)),
                      tgt_cls=np.ascontiguousarray(tgt_cls),
                      c_off=c_off, c_pred=preds.astype(np.int32),
                      c_emb=np.ascontiguousarray(c_emb.astype(np.float32)).reshape(n_c, dim),
                      scene_of_q=np.full(n_q, scene_id, np.int32),
                      planted=targets, planted_lm=lms)


# ---------------------------------------------------------------------------
# Named workloads.  Sizes follow the configurations the library is measured on.
# ---------------------------------------------------------------------------

def _room_n200(n_q=64):
    sc = make_scene(0, 200, 512, extent=(10.0, 10.0, 3.0), n_classes=16, n_views=4)
    qb = make_queries(100, sc, n_q, m_choices=(2,))
    return [sc], qb


def _site_n20k(n_q=4096, qseed=101):
    sc = make_scene(1, 20000, 1152, extent=(120.0, 120.0, 10.0), n_classes=400,
                    n_views=8, distractor_classes=20, distractor_frac=0.30)
    qb = make_queries(qseed, sc, n_q, m_choices=(1, 2, 3, 4),
                      distractor_classes=20, distractor_target_frac=0.5)
    return [sc], qb


def _multi_scene(n_scenes=67, n_q_total=44000, seed=2, n_lo=100, n_hi=20000):
    rng = np.random.Generator(np.random.PCG64(seed))
    ns = np.exp(rng.uniform(math.log(n_lo), math.log(n_hi), size=n_scenes)).astype(np.int64)
    scenes, parts = [], []
    per = [n_q_total // n_scenes + (1 if i < n_q_total % n_scenes else 0) for i in range(n_scenes)]
    for i, n in enumerate(ns):
        side = 120.0 * math.sqrt(n / 20000.0)
        height = min(max(side / 12.0, 3.0), 10.0)
        n_cls = max(16, int(round(400 * n / 20000)))
        n_dis = max(1, int(round(20 * n / 20000)))
        sc = make_scene(1000 + i, int(n), 1152, extent=(side, side, height), n_classes=n_cls,
                        n_views=8, distractor_classes=n_dis, distractor_frac=0.30)
        qb = make_queries(2000 + i, sc, per[i], m_choices=(0, 1, 2, 3, 4),
                          distractor_classes=n_dis, distractor_target_frac=0.5, scene_id=i)
        scenes.append(sc)
        parts.append(qb)
    return scenes, concat_batches(parts)


def _site_n100k(n_q=16384):
    sc = make_scene(4, 100000, 1152, extent=(300.0, 300.0, 15.0), n_classes=2000,
                    n_views=8, distractor_classes=100, distractor_frac=0.30)
    qb = make_queries(104, sc, n_q, m_choices=(1, 2, 3, 4),
                      distractor_classes=100, distractor_target_frac=0.5)
    return [sc], qb


# ---------------------------------------------------------------------------
# Several embedding spaces and query channels (App. D.2 step 3: four query
# channels over three embedding spaces; caption text, SigLIP2 image and
# Qwen3-VL image embeddings).  Space 0 is the scene's own descriptor array.
# ---------------------------------------------------------------------------

# (space, weight, noise multiplier) per channel, in the paper's order: the
# caption-text space queried with the target description (w = 1.0) and with
# the raw utterance (w = 0.5, a less specific phrase: twice the noise), the
# image space of the scene's descriptors (w = 0.75) and a second image space
# (w = 1.0).  Spaces: 0 = the scene's descriptors, 1 = text, 2 = second image.
PAPER_CHANNELS = ((1, 1.0, 1.0), (1, 0.5, 2.0), (0, 0.75, 1.0), (2, 1.0, 1.0))


@dataclasses.dataclass
class Spaces:
    desc: list                # per space [n, dim_s] float32, unit rows
    centroids: list           # per space [n_classes, dim_s] float64
    noise_sigma: list         # per space: per-dimension descriptor noise

    @property
    def dims(self):
        return [int(d.shape[1]) for d in self.desc]


def add_spaces(scene: Scene, seed: int, dims=(1024, 2048), noise_scale: float = 0.15) -> Spaces:
    """The scene's descriptors as space 0 plus one space per entry of `dims`:
    per space, unit Gaussian class centroids of its own and each object's
    descriptor = its class centroid + N(0, (noise_scale / sqrt(dim))^2),
    renormalised (the recipe of make_scene)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    n_classes = scene.centroids.shape[0]
    descs, cents, sigmas = [scene.desc], [scene.centroids], [scene.noise_sigma]
    for dim in dims:
        cen = _unit_rows(rng.standard_normal((n_classes, dim)))
        sg = noise_scale / math.sqrt(dim)
        d = _unit_rows(cen[scene.cls] + sg * rng.standard_normal((scene.n, dim))).astype(np.float32)
        descs.append(np.ascontiguousarray(d))
        cents.append(cen)
        sigmas.append(sg)
    return Spaces(desc=descs, centroids=cents, noise_sigma=sigmas)


@dataclasses.dataclass
class ChannelQueries:
    channels: list            # [(space, weight)]
    tgt: list                 # per channel [n_q, dim_space] float32
    lm: list                  # per channel [n_c, dim_space] float32


def channel_queries(seed: int, scene: Scene, spaces: Spaces, qb: QueryBatch, channels=PAPER_CHANNELS) -> ChannelQueries:
    """Per-channel target and landmark embeddings for the planted targets and
    landmarks of `qb`: channel c of space s draws its class centroid in s plus
    noise of (noise multiplier x the space's descriptor noise)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    tcls = scene.cls[qb.planted]
    lcls = scene.cls[qb.planted_lm] if qb.n_c else np.zeros(0, np.int64)
    tgt, lm = [], []
    for sp, _, mult in channels:
        cen, sg = spaces.centroids[sp], spaces.noise_sigma[sp] * mult
        dim = cen.shape[1]
        tgt.append(np.ascontiguousarray((cen[tcls] + sg * rng.standard_normal((qb.n_q, dim))).astype(np.float32)))
        lm.append(np.ascontiguousarray((cen[lcls] + sg * rng.standard_normal((qb.n_c, dim))).astype(np.float32)
                                       .reshape(qb.n_c, dim)))
    return ChannelQueries(channels=[(int(c[0]), float(c[1])) for c in channels], tgt=tgt, lm=lm)


# ---------------------------------------------------------------------------
# Mapping-side association (App. D.1 steps 3-5): the memory's entities as 3D
# Gaussians with appearance features and weights, and a batch of detections.
# ---------------------------------------------------------------------------

def _yaw_cov(sizes, yaw):
    """Packed covariances (xx, xy, xz, yy, yz, zz) of boxes of the given sizes
    (the moments of the uniform distribution over the box) turned by yaw."""
    v = (sizes ** 2) / 12.0
    c, s_ = np.cos(yaw), np.sin(yaw)
    xx = c * c * v[:, 0] + s_ * s_ * v[:, 1]
    yy = s_ * s_ * v[:, 0] + c * c * v[:, 1]
    xy = c * s_ * (v[:, 0] - v[:, 1])
    z = np.zeros_like(xx)
    return np.stack([xx, xy, z, yy, z, v[:, 2]]).astype(np.float32)


def make_association(seed: int, scene: Scene, n_det: int, feat_dim: int = 256, new_frac: float = 0.1,
                     bridge_frac: float = 0.05, inactive_frac: float = 0.05):
    """Entities: the scene's objects as Gaussians (box centre; box-moment
    covariance turned by a random yaw), a feat_dim appearance feature per
    object (its class's unit Gaussian centroid plus noise of norm about 0.15),
    a weight (1-20 fused detections) and an active flag.  Detections: mostly
    re-observations of random entities (centre moved by N(0, 0.05^2) m,
    sizes by 5%, yaw by 0.1 rad, feature re-drawn around the class centroid),
    a fraction placed midway between two same-class neighbours (a detection
    that bridges two entities) and a fraction of new objects."""
    rng = np.random.Generator(np.random.PCG64(seed))
    n = scene.n
    n_cls = int(scene.cls.max()) + 1
    cent = _unit_rows(rng.standard_normal((n_cls, feat_dim)))
    sg = 0.15 / math.sqrt(feat_dim)
    sizes = scene.box[3:].T.astype(np.float64)
    yaw = rng.uniform(0, np.pi, n)
    ent = dict(mu=scene.box[:3].astype(np.float32), cov=_yaw_cov(sizes, yaw),
               feat=_unit_rows(cent[scene.cls] + sg * rng.standard_normal((n, feat_dim))).astype(np.float32),
               w=rng.integers(1, 21, n).astype(np.float32),
               active=(rng.uniform(size=n) >= inactive_frac).astype(np.int32))
    kind = rng.uniform(size=n_det)
    src = rng.integers(0, n, n_det)
    mu = np.zeros((3, n_det)); sz = np.zeros((n_det, 3)); yw = np.zeros(n_det); cls = np.zeros(n_det, np.int64)
    from scipy.spatial import cKDTree
    centers = scene.box[:3].T.astype(np.float64)
    tree = cKDTree(centers)
    for d in range(n_det):
        e = int(src[d])
        if kind[d] < new_frac:
            ext = np.asarray(scene.extent if scene.extent[0] > 0 else centers.max(axis=0))
            mu[:, d] = rng.uniform(0, 1, 3) * ext
            sz[d] = rng.lognormal(-1.0, 0.5, 3)
            yw[d] = rng.uniform(0, np.pi)
            cls[d] = rng.integers(0, n_cls)
            continue
        cls[d] = scene.cls[e]
        if kind[d] < new_frac + bridge_frac:
            _, nb = tree.query(centers[e], k=min(8, n))
            same = [int(j) for j in np.atleast_1d(nb) if j != e and scene.cls[j] == scene.cls[e]]
            if same:
                mu[:, d] = 0.5 * (centers[e] + centers[same[0]])
                sz[d] = np.abs(centers[e] - centers[same[0]]) + 0.5 * (sizes[e] + sizes[same[0]])
                yw[d] = yaw[e]
                continue
        mu[:, d] = centers[e] + 0.05 * rng.standard_normal(3)
        sz[d] = sizes[e] * (1.0 + 0.05 * rng.standard_normal(3))
        yw[d] = yaw[e] + 0.1 * rng.standard_normal()
    det = dict(mu=mu.astype(np.float32), cov=_yaw_cov(np.abs(sz), yw),
               feat=_unit_rows(cent[cls] + sg * rng.standard_normal((n_det, feat_dim))).astype(np.float32))
    return ent, det


def concat_batches(parts):
    offs = [0]
    for p in parts:
        offs.append(offs[-1] + p.n_c)
    c_off = np.concatenate([[0]] + [p.c_off[1:].astype(np.int64) + o for p, o in zip(parts, offs)])
    return QueryBatch(
        tgt_emb=np.ascontiguousarray(np.concatenate([p.tgt_emb for p in parts])),
        tgt_cls=np.concatenate([p.tgt_cls for p in parts]),
        c_off=c_off.astype(np.int32),
        c_pred=np.concatenate([p.c_pred for p in parts]),
        c_emb=np.ascontiguousarray(np.concatenate([p.c_emb for p in parts])),
        scene_of_q=np.concatenate([p.scene_of_q for p in parts]),
        planted=np.concatenate([p.planted for p in parts]),
        planted_lm=np.concatenate([p.planted_lm for p in parts]),
    )


WORKLOADS = {
    # 10x10x3 m room, N=200, D=512, 16 classes, 4 views, 64 queries x 2 constraints
    "room_n200_d512": _room_n200,
    # 120x120x10 m site, N=20,000, D=1152, 400 classes (30% in 20 look-alike
    # classes), 8 views, 4,096 queries with 1-4 constraints
    "site_n20k_d1152": _site_n20k,
    # 67 scenes, N log-uniform in [100, 20,000], constant density, 44,000 queries, 0-4 constraints
    "multi67_d1152": _multi_scene,
    # the 20k site with 16,384 queries (reduced-precision study)
    "site_n20k_d1152_q16k": lambda: _site_n20k(n_q=16384, qseed=103),
    # 300x300x15 m site, N=100,000, D=1152, 16,384 queries
    "site_n100k_d1152": _site_n100k,
}


def workload(name: str, **kw):
    """Return (scenes, queries) for a named workload."""
    return WORKLOADS[name](**kw)
