"""GPU parity for the further predicates of App. D.2 step 4 (NextTo, On,
InFrontOf, Behind, Closest, Farthest, Inside) and the Hellinger form of Near
(Sec. 2.3) and the ternary Between (App. B) next to the first five, through
the C ABI, against the FP64 oracle
with the tie-tolerant checker.

Queries draw every constraint's predicate uniformly from all fifteen codes
(a Between takes two consecutive constraints);
the scenes are the room (200 objects, 4 views) and a slice of the
20,000-object site (8 views), plus a hand-built scene whose answer is fixed.
"""
import numpy as np
import pytest

from oracle import parity
import synth
from synth import QueryBatch

pytestmark = pytest.mark.gpu

ALL = list(range(15))


@pytest.fixture(scope="module")
def F():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    import paper_2606_15476_gb300 as F
    return F


@pytest.fixture(scope="module")
def ctx(F):
    c = F.farm_create(0)
    yield c
    F.farm_destroy(c)


def _run(F, ctx, qb, prec, k=10):
    h = F.farm_query_batch(ctx, qb.scene_of_q, qb.tgt_emb, qb.tgt_cls, qb.c_off, qb.c_pred, qb.c_emb, prec)
    return h, F.farm_topk(ctx, h, k, qb.n_q)


@pytest.mark.parametrize("prec", ["fp32", "fp32_simt"])
def test_room_every_predicate(F, ctx, prec):
    scenes, _ = synth.workload("room_n200_d512")
    sc = scenes[0]
    F.farm_memory_upload(ctx, 60, sc.desc, sc.cls, sc.box, sc.views)
    qb = synth.make_queries(600, sc, 96, m_choices=(1, 2, 3, 4), scene_id=60, preds=ALL)
    assert set(np.unique(qb.c_pred).tolist()) == set(ALL)
    code = {"fp32": F.PREC_FP32, "fp32_simt": F.PREC_FP32_SIMT}[prec]
    h, out = _run(F, ctx, qb, code)
    rep = parity.check_topk(sc, qb, 10, out["idx"], out["score"], out["pred"], out["anchor"])
    assert rep.ok(), rep.summary()
    t, l = F.farm_candidates(ctx, h, qb.n_q, qb.n_c)
    fails = parity.check_candidates(sc, qb, t, l)
    assert not fails, fails[:3]


def test_site_slice_every_predicate(F, ctx):
    scenes, _ = synth.workload("site_n20k_d1152")
    sc = scenes[0]
    F.farm_memory_upload(ctx, 61, sc.desc, sc.cls, sc.box, sc.views)
    qb = synth.make_queries(601, sc, 120, m_choices=(1, 2, 3, 4), distractor_classes=20,
                            distractor_target_frac=0.5, scene_id=61, preds=ALL)
    h, out = _run(F, ctx, qb, F.PREC_FP32)
    rep = parity.check_topk(sc, qb, 10, out["idx"], out["score"], out["pred"], out["anchor"])
    assert rep.ok(), rep.summary()


def test_reduced_precision_every_predicate(F, ctx):
    """BF16 with FP32 rescore gives the FP32 path's TopK (Recall@10 >= 0.99)."""
    scenes, _ = synth.workload("site_n20k_d1152")
    sc = scenes[0]
    F.farm_memory_upload(ctx, 61, sc.desc, sc.cls, sc.box, sc.views)
    qb = synth.make_queries(602, sc, 512, m_choices=(1, 2, 3, 4), scene_id=61, preds=ALL)
    _, ref = _run(F, ctx, qb, F.PREC_FP32)
    _, got = _run(F, ctx, qb, F.PREC_BF16)
    hits = sum(len(set(ref["idx"][q].tolist()) & set(got["idx"][q].tolist())) for q in range(qb.n_q))
    assert hits / (10.0 * qb.n_q) >= 0.99


def _hand_scene():
    """Two mugs; only mug 1 stands on the table (object 2); a lamp (object 3)
    stands 2 m from mug 1, on the side away from the table.  Descriptors:
    mugs e0 (mug 1 slightly off, so mug 0 ranks first), table e1, lamp e2."""
    centres = [[1.0, 1.0, 0.85], [3.0, 1.0, 0.85], [3.0, 1.2, 0.35], [3.0, -1.0, 0.85]]
    sizes = [[0.1, 0.1, 0.1], [0.1, 0.1, 0.1], [1.2, 0.8, 0.7], [0.3, 0.3, 1.0]]
    box = np.zeros((6, 4), np.float32)
    box[:3] = np.asarray(centres, np.float32).T
    box[3:] = np.asarray(sizes, np.float32).T
    d = np.zeros((4, 8), np.float32)
    d[0, 0] = d[1, 0] = 1.0
    d[1, 3] = 0.01           # the two mugs differ slightly: mug 0 ranks first semantically
    d[2, 1] = 1.0
    d[3, 2] = 1.0
    views = np.zeros((6, 1, 4), np.float32)     # one view per object, 2 m south, looking north
    views[0, 0] = box[0]
    views[1, 0] = box[1] - 2.0
    views[2, 0] = box[2]
    views[4, 0] = 1.0
    from synth import Scene
    return Scene(desc=d, cls=np.array([0, 0, 1, 2], np.int32), box=box, views=views)


@pytest.mark.parametrize("pred,expect", [(6, 1), (9, 1), (10, 0)])
def test_hand_built_scene(F, ctx, pred, expect):
    """'mug on the table' and 'mug closest to the lamp' pick mug 1 over the
    semantically preferred mug 0; 'mug farthest from the lamp' picks mug 0."""
    sc = _hand_scene()
    F.farm_memory_upload(ctx, 62, sc.desc, sc.cls, sc.box, sc.views)
    lm = {6: 1, 9: 2, 10: 2}[pred]     # landmark: table (e1) or lamp (e2)
    qb = QueryBatch(tgt_emb=np.eye(1, 8, dtype=np.float32), tgt_cls=np.array([0], np.int32),
                    c_off=np.array([0, 1], np.int32), c_pred=np.array([pred], np.int32),
                    c_emb=np.eye(1, 8, lm, dtype=np.float32), scene_of_q=np.array([62], np.int32))
    h, out = _run(F, ctx, qb, F.PREC_FP32, k=2)
    assert int(out["idx"][0, 0]) == expect
    rep = parity.check_topk(sc, qb, 2, out["idx"], out["score"], out["pred"], out["anchor"])
    assert rep.ok(), rep.summary()


def test_hand_built_inside(F, ctx):
    """'mug inside the table's box': with mug 1 lowered into the table's
    volume it is chosen over the semantically preferred mug 0 (which scores
    s_sem / 2 = 1/12 against mug 1's 1/7)."""
    sc = _hand_scene()
    sc.box[2, 1] = 0.35            # mug 1 now lies wholly inside the table's box
    F.farm_memory_upload(ctx, 63, sc.desc, sc.cls, sc.box, sc.views)
    qb = QueryBatch(tgt_emb=np.eye(1, 8, dtype=np.float32), tgt_cls=np.array([0], np.int32),
                    c_off=np.array([0, 1], np.int32), c_pred=np.array([12], np.int32),
                    c_emb=np.eye(1, 8, 1, dtype=np.float32), scene_of_q=np.array([63], np.int32))
    h, out = _run(F, ctx, qb, F.PREC_FP32, k=2)
    assert int(out["idx"][0, 0]) == 1 and int(out["anchor"][0, 0, 0]) == 2
    assert float(out["pred"][0, 0, 0]) == 1.0
    assert float(out["score"][0, 0]) == pytest.approx(1.0 / 7.0, rel=1e-6)
    rep = parity.check_topk(sc, qb, 2, out["idx"], out["score"], out["pred"], out["anchor"])
    assert rep.ok(), rep.summary()


@pytest.mark.parametrize("prec", ["fp32", "fp32_simt"])
def test_between_pairs(F, ctx, prec):
    """Queries made mostly of Between pairs (with Above / Near beside them)."""
    scenes, _ = synth.workload("room_n200_d512")
    sc = scenes[0]
    F.farm_memory_upload(ctx, 64, sc.desc, sc.cls, sc.box, sc.views)
    qb = synth.make_queries(605, sc, 96, m_choices=(2, 3, 4), scene_id=64, preds=[13, 13, 0, 4])
    assert int(np.sum(qb.c_pred == 13)) >= 40
    code = {"fp32": F.PREC_FP32, "fp32_simt": F.PREC_FP32_SIMT}[prec]
    h, out = _run(F, ctx, qb, code)
    rep = parity.check_topk(sc, qb, 10, out["idx"], out["score"], out["pred"], out["anchor"])
    assert rep.ok(), rep.summary()
    # a malformed pair is rejected before anything runs
    bad = qb.subset(range(4))
    bad.c_pred[:] = 14
    with pytest.raises(F.FarmError):
        _run(F, ctx, bad, code)
