"""Hand-built scenes for the tests (layout only; no method arithmetic)."""
import json
import os

import numpy as np

from synth import QueryBatch, Scene

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
PRED_CODE = {"above": 0, "below": 1, "left_of": 2, "right_of": 3, "near": 4}


def load_golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def south_view_scene(objects, dim):
    """Scene with one stored view per object, 2 m south looking north."""
    n = len(objects)
    desc = np.array([o["desc"] for o in objects], dtype=np.float64)
    desc = (desc / np.linalg.norm(desc, axis=1, keepdims=True)).astype(np.float32)
    cls = np.array([o["cls"] for o in objects], dtype=np.int32)
    box = np.zeros((6, n), np.float32)
    for j, o in enumerate(objects):
        box[:3, j] = o["center"]
        box[3:, j] = o["size"]
    views = np.zeros((6, 1, n), np.float32)
    views[0, 0] = box[0]
    views[1, 0] = box[1] - 2.0
    views[2, 0] = box[2]
    views[4, 0] = 1.0
    assert desc.shape[1] == dim
    return Scene(desc=desc, cls=cls, box=box, views=views)


def single_query(tgt_emb, tgt_cls, preds, lm_embs, dim):
    m = len(preds)
    return QueryBatch(
        tgt_emb=np.asarray(tgt_emb, np.float32).reshape(1, dim),
        tgt_cls=np.array([tgt_cls], np.int32),
        c_off=np.array([0, m], np.int32),
        c_pred=np.asarray(preds, np.int32).reshape(m),
        c_emb=np.asarray(lm_embs, np.float32).reshape(m, dim),
        scene_of_q=np.zeros(1, np.int32))


def golden_case(g, which):
    """(scene, query batch, params dict) for one constraint subset of the worked scene."""
    sc = south_view_scene(g["objects"], g["dim"])
    cons = g["query"]["constraints"]
    keep = {"both": [0, 1], "below_only": [0], "left_of_only": [1], "none": []}[which]
    preds = [PRED_CODE[cons[i]["pred"]] for i in keep]
    lms = [cons[i]["landmark_emb"] for i in keep]
    qb = single_query(g["query"]["target_emb"], g["query"]["target_cls"], preds,
                      np.array(lms, np.float32).reshape(len(keep), g["dim"]), g["dim"])
    return sc, qb


def tiny_scene(rng, n, dim, n_views=2, extent=(6.0, 6.0, 3.0), n_classes=3):
    """Random small scene with views on a partial arc (used by brute-force checks)."""
    centers = rng.uniform(0, 1, size=(n, 3)) * np.asarray(extent)
    desc = rng.standard_normal((n, dim))
    desc = (desc / np.linalg.norm(desc, axis=1, keepdims=True)).astype(np.float32)
    cls = rng.integers(0, n_classes, size=n).astype(np.int32)
    box = np.concatenate([centers.T, rng.uniform(0.1, 1.0, size=(3, n))]).astype(np.float32)
    views = np.zeros((6, n_views, n), np.float32)
    phase = rng.uniform(0, 2 * np.pi, size=n)
    for v in range(n_views):
        th = phase + 0.6 * v
        views[0, v] = centers[:, 0] + 2 * np.cos(th)
        views[1, v] = centers[:, 1] + 2 * np.sin(th)
        views[2, v] = centers[:, 2] + rng.uniform(-0.3, 0.3, size=n)
        views[3, v] = -np.cos(th)
        views[4, v] = -np.sin(th)
    return Scene(desc=desc, cls=cls, box=box, views=views)
